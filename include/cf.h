/*
 * cf.h -- C ABI of cfgpu, exact cell-list pair counting on NVIDIA GB300 (sm_103a).
 *
 * The operation is the pair-separation histogram of Sinha & Garrison,
 * "Corrfunc: blazing fast correlation functions with AVX512F SIMD intrinsics"
 * (arXiv:1911.08275):
 *   - Sec. 1.1, Code 1: for every pair (i, j) compute a separation, skip it
 *     unless Rmin <= sep < Rmax, and add one (and a weight) to its bin;
 *   - Sec. 1.1, Eq. "separations": xi(r) uses r = |x_j - x_i|; wp(rp) uses
 *     rp = |(dx, dy)| and pi = |dz| with the extra filter pi < pimax;
 *   - Sec. 1.2 and 2.1: points are gridded into cells so only neighbouring
 *     cells are searched, sorted along z, and auto-correlations visit each
 *     unordered cell pair once and double the counts;
 *   - Sec. 2.2: cell pairs whose bounding boxes are >= Rmax apart are pruned;
 *   - Sec. 2.2, Code 3/4: separations are compared squared against squared
 *     bin edges; no square root or logarithm decides a bin.
 *
 * Exactness.  Every count is defined by canonical IEEE binary64 arithmetic
 * (inputs promoted exactly to double, no fused multiply-add):
 *   dx = x_j - x_i; periodic: if dx > L/2: dx -= L; elif dx < -L/2: dx += L;
 *   rp2 = dx*dx + dy*dy;  r2 = rp2 + dz*dz;  bin k iff e_k^2 <= r2 < e_{k+1}^2;
 *   pi bins [P_m, P_{m+1}) with P_m = (pimax*m)/npibins, P_npibins = pimax.
 * CF_MODE_FP64 evaluates exactly that.  CF_MODE_FP32_RECHECK evaluates the
 * distances in float32 and re-evaluates in binary64 every pair whose float32
 * value lies within a proven error bound of a bin edge, Rmin, Rmax or a pi
 * edge; its integer counts are therefore identical to CF_MODE_FP64.
 *
 * Conventions shared by all entry points:
 *   - Return value: CF_OK (0) or a negative CF_E* status; the entry points
 *     never throw, abort or exit.  cf_last_error() describes the last failure
 *     of the calling thread.
 *   - Auto-correlation counts ordered pairs i != j (each unordered pair twice);
 *     cross-correlation counts every (i in d1, j in d2).
 *   - Inputs are borrowed for the duration of the call.  Position arrays may
 *     live in device memory (used in place) or host memory (copied to the
 *     device inside the call; page-locked host memory copies fastest).
 *   - Results are written to caller-owned HOST arrays before the call returns
 *     (the call synchronises its stream).
 *   - Scratch memory comes from the stream-ordered allocator of the current
 *     device (cudaMallocAsync on cfg->stream) and is released before return.
 *   - Periodic mode requires coordinates in [0, boxsize) per axis and
 *     Rmax, pimax < boxsize/2 (so the minimum image is unique).
 */
#ifndef CFGPU_CF_H
#define CFGPU_CF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CF_OK 0
#define CF_EINVAL (-1)    /* invalid argument (see cf_last_error)               */
#define CF_ENOMEM (-2)    /* device or host allocation failed                   */
#define CF_ECUDA (-3)     /* a CUDA runtime call failed                         */
#define CF_ETIMEOUT (-4)  /* a bounded device-side wait gave up (after ~2 s;
                             the kernel returns, the context stays usable)      */
#define CF_EDEVICE (-5)   /* a kernel reported an inconsistency (error word)    */

typedef enum { CF_FLOAT32 = 0, CF_FLOAT64 = 1 } cf_dtype;

typedef enum {
    CF_MODE_FP64 = 0,          /* all distance arithmetic in binary64          */
    CF_MODE_FP32_RECHECK = 1   /* float32 bulk + binary64 re-check near edges   */
} cf_mode;

/* Flags (cf_config.flags). */
#define CF_FLAG_COUNT_EVALS (1u << 0) /* count pair evaluations into n_evaluated */
#define CF_FLAG_NO_PRUNE (1u << 1)    /* disable bounding-box cell-pair pruning   */
#define CF_FLAG_VERIFY_BAND (1u << 2) /* FP32 mode: also evaluate every pair in
                                         binary64 and count float32 decisions that
                                         disagree into n_band_violations (debug)  */
#define CF_FLAG_DEBUG_STALL (1u << 3) /* diagnostic (float32 DD(r) without sums):
                                         each CTA's first tile barrier is armed for
                                         a copy that is never issued, and the waits
                                         give up after 1 ms, so the call returns
                                         CF_ETIMEOUT; tests the bounded waits.
                                         Ignored by the other kernels.          */

/* One catalogue: n points with coordinates x[i], y[i], z[i] of type
 * cf_config.dtype, contiguous, in device or host memory, and optional float64
 * weights w[i] (same memory kind as x) or NULL. */
typedef struct {
    const void *x, *y, *z;
    const double *w;
    int64_t n;
} cf_catalog;

typedef struct {
    int periodic;        /* 1: periodic box [0, boxsize)^3; 0: open box          */
    double boxsize[3];   /* box side per axis (periodic only)                     */
    cf_dtype dtype;      /* element type of x, y, z                               */
    cf_mode mode;        /* arithmetic path                                       */
    int weighted;        /* 1: accumulate w_i * w_j per bin (weights required)   */
    int want_ravg;       /* 1: accumulate the mean separation per bin             */
    int refine[3];       /* cell refinement (rx, ry, rz); {0,0,0} = automatic:
                            (r, r, 1) with r = round(Rmax / s) in [1, 4], s the
                            column side over which the smaller catalogue holds
                            about 1024 points.  Columns in
                            x, y are >= Rmax/rx wide (Sec. 3.1 names (2, 2, 1)
                            as a good start); rz sets the z-cell granularity of
                            the in-column sort.                                  */
    uint32_t flags;      /* CF_FLAG_*                                             */
    void *stream;        /* cudaStream_t to run on; NULL = legacy default stream  */
    int autotune;        /* 1: choose refine (and the float32 DD(r) kernel shape)
                            by timing candidates (the automatic r and r +- 1,
                            then the kernel shapes) once per problem signature and
                            caching the winner (Sec. 3.1 asks for an automatic
                            choice of the refinement); fields set explicitly
                            (refine != {0,0,0}, pair_chunk, pair_pp) are kept.   */
    int pair_chunk;      /* float32 DD(r) kernel: primary lanes per warp chunk
                            (8, 16 or 32 with pair_pp 1; 8 or 16 with pair_pp 2,
                            32 runs as 16; 8 with pair_pp 4); 0 = default 16      */
    int pair_pp;         /* float32 kernels: primaries per lane, DD(r) 1, 2 or 4,
                            DD(rp, pi) 2 (else one, with pair_chunk lanes);
                            0 = default 2                                         */
    int shard_index;     /* with shard_count > 1: count only the column pairs
                            whose primary column starts in slice shard_index of
                            shard_count equal slices of the gridded d1 points;  */
    int shard_count;     /* the shards' histograms sum to the full one (one shard
                            per process / GPU).  0 or 1 = no sharding.            */
} cf_config;

/* Caller-owned host outputs.  Arrays are NULL when not wanted. */
typedef struct {
    uint64_t *npairs;    /* [nbins] (xi) or [n_rp_bins * npibins] rp-major      */
    double *wsum;        /* same shape: sum of w_i*w_j (weighted) else unused     */
    double *ravg;        /* same shape: mean separation (r or rp), weighted by
                            w_i*w_j when weighted; 0 for empty bins.  Binary64
                            mode: exact per-pair terms, sums within 1e-12
                            relative (summation order).  Float32 mode: r from
                            the float32 squared distance corrected with the
                            coordinates' float32 rounding residuals (~3e-7
                            relative per pair); DD(r) terms rounded to a fixed-
                            point grid scaled by the largest weights (2^-22
                            max|w w| / |w w| relative per term), so wsum and
                            ravg agree to 1e-5 relative for weights within a
                            factor 3 of each other                              */
    uint64_t n_cellpairs;       /* column pairs kept after pruning                */
    uint64_t n_evaluated;       /* pair evaluations (CF_FLAG_COUNT_EVALS)        */
    uint64_t n_rechecked;       /* pairs re-evaluated in binary64 (FP32 mode)    */
    uint64_t n_band_violations; /* CF_FLAG_VERIFY_BAND: must be 0                 */
    double kernel_ms;           /* device time of the pair kernel                 */
    double total_ms;            /* device time of the whole call                  */
    uint64_t n_kernels;         /* kernels the call launched (gridding, bounding
                                   box, work list, pair kernel; copies and memsets
                                   excluded)                                      */
    int refine_used[3];         /* refinement the call used                        */
    int chunk_used, pp_used;    /* float32 DD(r) kernel shape the call used        */
    int tuned;                  /* 0 no autotuning, 1 this call tuned (timed the
                                   candidates, then counted with the winner),
                                   2 the cached choice was used                   */
    int table_linear;           /* float32 paths: 1 if the bin table's cells are
                                   linear in d2, 0 if logarithmic                 */
} cf_result;

/*
 * DD(r) for xi(r) (Sec. 1.1 Code 1 with the xi separation of Eq.
 * "separations"; bins tested on squares as in Sec. 2.2 Code 4).
 *   autocorr   1: pairs within d1 (d2 ignored, may be NULL); 0: d1 x d2.
 *   edges      nedges >= 2 strictly increasing bin edges, edges[0] >= 0,
 *              host memory; bins k = [edges[k], edges[k+1]), nbins = nedges-1
 *              <= 64; Rmin = edges[0], Rmax = edges[nedges-1].
 *   res        npairs[nbins] (required), wsum[nbins], ravg[nbins] (optional).
 * Errors: CF_EINVAL for bad arguments (NULL pointers, n < 0, n >= 2^31, edges
 * not increasing, nbins > 64, weighted without weights, periodic with
 * Rmax >= boxsize/2 or a coordinate outside [0, boxsize) or non-finite).
 */
int cf_countpairs_xi(int autocorr, const cf_catalog *d1, const cf_catalog *d2,
                     const double *edges, int nedges, const cf_config *cfg, cf_result *res);

/*
 * DD(rp, pi) for wp(rp) (Sec. 1.1 Eq. "separations", rp-pi case; the line of
 * sight is z; Sec. 2.1 sizes cells by Rmax in x, y and by pimax in z).
 *   rp_edges   n_rp_edges >= 2 increasing edges on rp (host), <= 64 rp bins.
 *   pimax      > 0; pairs count only if |dz| < pimax.
 *   npibins    >= 1 pi bins [P_m, P_{m+1}), P_m = (pimax*m)/npibins; at most
 *              4096 bins in total (n_rp_bins * npibins).
 *   res        npairs[n_rp_bins * npibins], rp-major (index k*npibins + m).
 *              Summing over m gives the paper's 1-D wp pair count.
 * Errors as cf_countpairs_xi, plus CF_EINVAL for pimax >= boxsize[2]/2 in
 * periodic mode.
 */
int cf_countpairs_rp_pi(int autocorr, const cf_catalog *d1, const cf_catalog *d2,
                        const double *rp_edges, int n_rp_edges, double pimax, int npibins,
                        const cf_config *cfg, cf_result *res);

/*
 * Allocation-free DD(r).  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory at call time -- for example a
 * process whose GPU memory is already reserved by another allocator, or a loop
 * that must never wait on cudaMalloc.  Same arguments and results as
 * cf_countpairs_xi, with these differences:
 *   - all device scratch comes from one static device array of 32 MiB inside
 *     the library (held by every GPU that loads it until the process exits);
 *     nothing is allocated or freed by the call;
 *   - each catalogue has at most 131072 points (CF_EINVAL above that).  When
 *     the grid the planner would choose does not fit the array (mostly the
 *     column-pair list of fine grids), the call plans coarser columns and
 *     z-cells until it fits; the counts do not depend on the grid;
 *   - coordinates must already be in device memory; no weights, no ravg;
 *     CF_FLAG_VERIFY_BAND is ignored; kernel_ms and total_ms are reported as 0;
 *   - the first call in each CUDA context (the first call on a device, and
 *     again after a device reset) looks up the array's device address with
 *     cudaGetSymbolAddress while that device is current: make that first call
 *     before any stream capture.  Every call synchronises cfg->stream (twice
 *     for open boxes) and returns CF_EINVAL if that stream is being captured;
 *   - every call on a device reuses the same array: calls whose GPU work
 *     overlaps (concurrent streams or threads) race and must be serialised.
 */
int cf_countpairs_xi_noalloc(int autocorr, const cf_catalog *d1, const cf_catalog *d2,
                             const double *edges, int nedges, const cf_config *cfg,
                             cf_result *res);

/*
 * Batched counting (a persistent launch over many jobs).  Jobs -- catalogues
 * of uneven sizes, DD(r) or DD(rp, pi), float32+re-check or binary64, auto or
 * cross, periodic or open -- are added to a batch and then run together: every
 * gridding stage runs once for all catalogues of all jobs (each catalogue a
 * segment of the launch), the work lists of all jobs in one more launch, and
 * one persistent kernel pulls column pairs from a single queue over all jobs'
 * work lists (the GPU analogue of the paper's OpenMP loop over cell pairs,
 * Sec. 2.1): a run is 16 launches whatever the number of jobs.  With
 * use_graph the whole sequence is captured once into a CUDA graph and replayed
 * by later runs.  A job's res->n_kernels is 0 (the launches are shared; the
 * batch's count is in cf_batch_stats).
 *   cf_batch_add_xi / cf_batch_add_rp_pi: arguments as cf_countpairs_xi /
 *     cf_countpairs_rp_pi, validated at once.  Batched jobs count unweighted
 *     pairs (cfg->weighted and cfg->want_ravg must be 0) and take coordinates
 *     in DEVICE memory; flags other than CF_FLAG_NO_PRUNE are ignored.  With
 *     cfg->autotune a job uses the tuner's refinement and, for float32 DD(r),
 *     kernel shape (16 x 2, 8 x 2, 16 x 1 or 32 x 1) for its signature; a
 *     signature the cache does not hold is tuned when the batch is planned, by
 *     timing the candidates with single calls as cf_countpairs_xi does (res
 *     reports refine_used, chunk_used, pp_used and tuned).  Without autotune a
 *     job uses its own refinement and the shape 16 x 2.
 *     The catalogues and res stay borrowed until cf_batch_destroy; their
 *     contents may change between runs.  A job's results are written to its
 *     res by every cf_batch_run (res takes the place of a separate result
 *     query).
 *   cf_batch_run: plans the jobs on the first run (open boxes: one bounding-box
 *     pass with a host synchronisation), counts every job and writes each
 *     job's res before returning (one synchronisation of the stream).  Later
 *     runs reuse the plan, and with use_graph replay the captured graph; an
 *     open-box job whose bounding box changed makes the run plan and capture
 *     again.  stream NULL runs on a stream owned by the batch.  stats may be
 *     NULL.  Errors name the job index in cf_last_error(); a failed job leaves
 *     every res of that run undefined.
 *   cf_batch_destroy: frees the batch's device memory, stream and graph.
 */
typedef struct cf_batch cf_batch;

typedef struct {
    uint64_t n_jobs;
    uint64_t n_kernels;   /* kernels of one run (gridding, work lists, offsets, batched kernel) */
    uint64_t pairs;       /* sum over jobs of the counted pairs                   */
    int used_graph;       /* 1 if the run launched the captured graph             */
    int planned;          /* 1 if the run (re)planned the jobs                    */
    int blocks;           /* CTAs of the batched kernel                           */
    double kernel_ms;     /* device time of the batched pair kernel (-1 when the
                             run replayed a graph: only the whole run is timed)  */
    double total_ms;      /* device time of the run (memsets to the final copy)   */
} cf_batch_stats;

int cf_batch_create(cf_batch **out);
int cf_batch_add_xi(cf_batch *b, int autocorr, const cf_catalog *d1, const cf_catalog *d2,
                    const double *edges, int nedges, const cf_config *cfg, cf_result *res);
int cf_batch_add_rp_pi(cf_batch *b, int autocorr, const cf_catalog *d1, const cf_catalog *d2,
                       const double *rp_edges, int n_rp_edges, double pimax, int npibins,
                       const cf_config *cfg, cf_result *res);
int cf_batch_run(cf_batch *b, void *stream, int use_graph, cf_batch_stats *stats);
int cf_batch_destroy(cf_batch *b);

/*
 * Autotuner cache (Sec. 3.1 leaves the refinement to the user and asks for an
 * automatic choice).  Entries map a problem signature -- kind, mode, dtype,
 * auto/cross, periodic, weighted, half-octave buckets of N1, N2 and of the
 * mean neighbour count within Rmax, number of bins -- to the refinement and
 * kernel shape that timed fastest.  The cache lives in host memory of the
 * process (shared by all threads); with the environment variable
 * CF_TUNE_CACHE=<path> it is loaded from that JSON file on first use and
 * written back after every new entry.
 *   cf_tune_save/cf_tune_load: write / merge a JSON file ({"version": 1,
 *     "entries": [{"key", "refine", "chunk", "pp", "ms"}, ...]}).  CF_EINVAL
 *     for an unreadable or malformed file (the cache is left unchanged).
 *   cf_tune_clear: drop every entry.   cf_tune_count: number of entries.
 * None of these touch the GPU.
 */
int cf_tune_save(const char *path);
int cf_tune_load(const char *path);
int cf_tune_clear(void);
int cf_tune_count(void);

/*
 * Float32 decision tables, for diagnostics and tests (host only: no device
 * work).  The float32 paths compute a squared separation d2~ in float32, bin
 * it with a byte table and settle what the table cannot with thresholds, so
 * that the counts equal the binary64 definition (bins [e_k, e_{k+1}) tested on
 * squares, Sec. 2.2):
 *   thr[0 .. 2 nedges): lo_0, hi_0, ..., lo_B, hi_B around E2_k = edges[k]^2
 *     (binary64), lo_k <= E2_k <= hi_k: d2~ < lo_k proves d2 < E2_k and
 *     d2~ >= hi_k proves d2 >= E2_k, for float32 coordinates of magnitude
 *     <= coord_max, a periodic shift of magnitude <= shift_max added to the
 *     primary in float32, and separations up to rmax; ncomp = 3 for 3-D
 *     separations, 2 for projected rp.
 *   table[0 .. lut_n): the entry of cell q is bin k when every value of the
 *     cell lies in [hi_k, lo_{k+1}), nedges - 1 when every value is surely
 *     not counted, 255 otherwise.  Value v >= 0 lies in cell
 *     round(v * lscale) (lin = 1; the float32 product rounded half to even)
 *     or ((bits(v) >> shift) - u0) mod 2^32 (lin = 0); cells past lut_n - 1
 *     (and NaN) use entry lut_n - 1.
 * thr holds 2 * nedges floats; table holds CF_BIN_TABLE_MAX bytes; info gets
 * the cell parameters.  Errors: CF_EINVAL for NULL pointers, fewer than 2 or
 * more than 65 edges, edges not finite, negative or not increasing, ncomp
 * not 2 or 3, and bounds that are negative or not finite.
 */
#define CF_BIN_TABLE_MAX 16384
typedef struct {
    int nthr;        /* thresholds written: 2 * nedges            */
    int lut_n;       /* table entries written                     */
    int lin;         /* 1: linear cells, 0: float-bit cells        */
    float lscale;    /* linear cells: cell = round(v * lscale)     */
    int shift;       /* float-bit cells: (bits(v) >> shift) - u0   */
    unsigned u0;
} cf_bin_tables;
int cf_debug_bin_tables(const double *edges, int nedges, int ncomp, double coord_max,
                        double shift_max, double rmax, float *thr, unsigned char *table,
                        cf_bin_tables *info);

/*
 * The pi-bin decision of the float32 DD(rp, pi) path, for diagnostics and
 * tests (host only).  With pscale = fl32(npibins / pimax) a pair's
 * t' = fl32(|dz~| * pscale - 1/2) (one rounding) gives m = round(t') (half to
 * even); the kernels trust bin m (not counted for m >= npibins) when
 * |t' - m| <= pband and re-check the pair in binary64 otherwise (pband = -1:
 * always).  Bounds as for cf_debug_bin_tables.  Errors: CF_EINVAL for NULL
 * pointers, pimax not positive and finite, npibins < 1, bounds negative or not
 * finite.
 */
int cf_debug_pi_band(double pimax, int npibins, double coord_max, double shift_max,
                     float *pscale, float *pband);

/* Text of the last non-zero status returned on the calling thread. */
const char *cf_last_error(void);

/* Library version string. */
const char *cf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CFGPU_CF_H */
