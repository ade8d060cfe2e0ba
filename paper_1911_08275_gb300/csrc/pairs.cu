// Pair kernels: the hot loop of cell-list pair counting (arXiv:1911.08275,
// Sec. 2.2: late entry / early exit on the z-sorted axis, Code 2; distance
// masks on squared separations, Code 3; histogram update by comparing against
// squared edges, Code 4), re-designed for GB300.
//
// Work unit = one (primary column a, secondary column b, periodic image) pair
// ("column pair"); columns are z-sorted (grid.cu).  The work-list kernel keeps
// the pairs whose bounding boxes are less than Rmax apart in (x, y) (Sec. 2.2)
// with their z reach.  A persistent CTA pulls kept pairs from a global counter,
// stages column b into shared memory with 1-D TMA bulk copies (cp.async.bulk +
// mbarrier, bounded waits) in tiles, and its 8 warps claim chunks of
// z-consecutive points of column a from a shared counter.  For each chunk and
// periodic z image a warp finds, by a lane-parallel search of the staged z
// values, the window of b points whose z can be within the reach of the chunk
// (the paper's late entry and early exit, applied per chunk rather than per
// particle), then sweeps it.
//
// Float32 DD(r) (Xi32Path; k_pipe with two tile buffers so that no CTA-wide
// barrier separates work items).  Each lane holds PP primaries, each broadcast
// into both halves of a 64-bit register, and evaluates them against two
// consecutive secondaries per 8-byte shared load with the sm_100-family packed
// f32x2 instructions.  The squared distance indexes (clamped, branch-free) a
// byte table built on the host from float32 thresholds lo_k < e_k^2 < hi_k that
// bracket every squared edge by a proven error bound; a safe cell gives the bin
// row, out-of-range distances a dummy row, and every lane adds one to its own
// column of the CTA's shared histogram with a shared-memory atomic (no bank
// conflicts, no branch).  A pair in a flagged cell (touching a band) sets a bit
// of the lane's mask; once per 8 steps a warp-uniform test hands the recorded
// pairs to a resolver that compares them with the thresholds and re-evaluates a
// distance inside a band with the canonical binary64 formula from the binary64
// copies of the two points, so counts are bit-identical to the binary64
// definition.  Float32 DD(rp, pi) (Rppi32PathPP) has the same structure with a
// 2-D histogram and a pi bin from one rounding.
//
// Binary64 kernels (Xi64Path, Rppi64Path, CF_MODE_FP64): the same traversal on
// binary64 copies with the canonical formula and exact squared-edge compares.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "cf_internal.cuh"
#include "pairs.cuh"

namespace cf {

// Rows of one float32 DD(rp, pi) histogram copy: the row that pairs in a flagged
// rp cell land in until they are settled (row -1, never read), the bins and the
// not-counted row, so a sign-extended table entry is a row index without a
// clamp.  Row 0 is the copy's second row.
inline __host__ __device__ int rppi32_rows(int nb) { return nb + 2; }

void plan_pairs(PairParams &P, PairLaunch &L)
{
    const int nb = P.nbins, nr = nb + 1;
    P.acc_off = 0;
    if (P.kind == 0) {
        L.hist_words = WARPS * nr * 32;  // per-lane rows + one dummy row per warp
        P.hcopies = WARPS;
        if (L.f64) {
            const Smem64 S = smem64_layout(P.tile_max, nb, 0, L.hist_words);
            P.hist_off = S.hist;
            P.acc_off = S.total;  // [warp][bin][w, r w] binary64 when weighted
            L.smem = P.wacc ? align_up(S.total + WARPS * nb * 16, 128) : S.total;
        } else if (P.wacc) {
            // count rows, then w and / or r w rows ([warp][row][lane] u32), then the
            // per-row scales of r w
            const int planes = 1 + (P.weighted ? 1 : 0) + (P.want_r ? 1 : 0);
            P.hist_off = XI32_HIST_OFF;
            L.hist_words = planes * WARPS * (nb + 2) * 32;
            L.smem = align_up(XI32_HIST_OFF + L.hist_words * 4 + (nb + 2) * 4, 128);
        } else if (L.pipe) {
            // one histogram copy shared by all warps, then the second tile buffer
            L.hist_words = (nb + 2) * 32;
            P.hist_off = XI32_HIST_OFF;
            L.smem = pipe_slot1_off(nb) + 3 * XI32_TSTRIDE;
        } else {
            L.hist_words = WARPS * (nb + 2) * 32;  // + a row for flagged table cells
            P.hist_off = XI32_HIST_OFF;
            L.smem = align_up(XI32_HIST_OFF + L.hist_words * 4, 128);
        }
        return;
    }
    // rp-pi: one histogram copy per warp while the CTA stays small enough for
    // three CTAs per SM, else fewer copies shared by several warps.
    const int copy = (L.f64 ? nr : rppi32_rows(nb)) * (P.npibins + 1);
    const int base = L.f64 ? smem64_layout(P.tile_max, nb, P.npibins, 0).hist
                           : align_up(RPPI_P_OFF + (P.npibins + 1) * 8, 128);
    const int per = copy * 4 + (P.wacc ? copy * 16 + 16 : 0);
    int hc = 1;
    for (int c = WARPS; c >= 1; c >>= 1)
        if (base + c * per <= 75 * 1024) {
            hc = c;
            break;
        }
    P.hcopies = hc;
    P.hist_off = base;
    L.hist_words = hc * copy;
    P.acc_off = align_up(base + L.hist_words * 4, 16);
    L.smem = align_up(P.wacc ? P.acc_off + hc * copy * 16 : base + L.hist_words * 4, 128);
}

namespace {

typedef unsigned long long u64;

__device__ __forceinline__ int floor_div(int a, int n)
{
    return a >= 0 ? a / n : -((-a + n - 1) / n);
}

// ---------------------------------------------------------------- packed f32x2
__device__ __forceinline__ u64 pack2(float lo, float hi)
{
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(u64 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 fsub2(u64 a, u64 b)
{
    u64 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 fmul2(u64 a, u64 b)
{
    u64 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 ffma2(u64 a, u64 b, u64 c)
{
    u64 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// ---------------------------------------------------------------- searches
// First index p in [0, n) with key(p) >= v (upper = false) or key(p) > v
// (upper = true); n if none.  Keys must be sorted.  All lanes call it with the
// same arguments; each round probes 32 positions.
template <class Key, class V>
__device__ __forceinline__ int warp_bound(Key key, int n, V v, bool upper, int lane)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int s = (hi - lo + 31) >> 5;
        const int p = lo + lane * s;
        bool q = false;
        if (p < hi) {
            const V z = key(p);
            q = upper ? (z <= v) : (z < v);
        }
        const int c = __popc(__ballot_sync(FULL, q));
        if (c == 0)
            break;
        const int nlo = lo + (c - 1) * s + 1;
        hi = min(hi, lo + c * s);
        lo = nlo;
    }
    return lo;
}

// Bin of a binary64 squared separation: k with E2[k] <= r2 < E2[k+1], else -1.
// Non-negative doubles order like their bit patterns, so integer compares suffice.
__device__ __forceinline__ int bin_f64(double r2, const double *E2, int nb)
{
    const long long u = __double_as_longlong(r2);
    const long long *e = reinterpret_cast<const long long *>(E2);
    if (!(u >= e[0] && u < e[nb]))
        return -1;
    int lo = 0, hi = nb;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (e[mid] <= u)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ double canon_r2(const double4_32a &p, const double4_32a &q, double Sx,
                                           double Sy, double Sz)
{
    const double dx = canon_comp(p.x, q.x, Sx);
    const double dy = canon_comp(p.y, q.y, Sy);
    const double dz = canon_comp(p.z, q.z, Sz);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// The same for an image whose shifts are all zero (canon_comp's adds are then
// skipped, so the value is bit-identical).  The binary64 sweeps choose between
// the two once per window: a shift test inside the pair loop is compiled into
// adds issued under a predicate, which still occupy the narrow binary64 pipe.
__device__ __forceinline__ double plain_r2(const double4_32a &p, const double4_32a &q)
{
    const double dx = __dsub_rn(q.x, p.x), dy = __dsub_rn(q.y, p.y), dz = __dsub_rn(q.z, p.z);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Binary64 re-evaluation of one pair inside an error band: bin row or -1.
__device__ __noinline__ int recheck64(const double *E2, int nb, const double4_32a *pa,
                                      const double4_32a *pb, int i, int j, double Sx, double Sy,
                                      double Sz)
{
    return bin_f64(canon_r2(pa[i], pb[j], Sx, Sy, Sz), E2, nb);
}

// Debug: does the float32 decision for d2 agree with binary64?  (1 = violation)
__device__ __noinline__ int verify_pair(float d2, const float *thr, int nthr, int nb,
                                        const double *E2, const double4_32a *pa,
                                        const double4_32a *pb, int i, int j, double Sx, double Sy,
                                        double Sz)
{
    int c = 0;
    while (c < nthr && thr[c] <= d2)
        ++c;
    if (c & 1)
        return 0;  // inside a band: re-checked, no float32 claim
    const int k32 = (c >= 2 && c <= 2 * nb) ? (c - 2) >> 1 : -1;
    const int k64 = bin_f64(canon_r2(pa[i], pb[j], Sx, Sy, Sz), E2, nb);
    return k32 != k64;
}

__device__ __forceinline__ u64 warp_sum_u64(u64 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Move one warp's per-lane counts to the global histogram (overflow guard).
__device__ void warp_flush(uint32_t *hw, int nb, unsigned long long *ghist, int lane)
{
    for (int b = 0; b < nb; ++b) {
        const u64 v = warp_sum_u64(hw[b * 32 + lane]);
        hw[b * 32 + lane] = 0u;
        if (lane == 0 && v)
            atomicAdd(&ghist[b], v);
    }
}

// The same for a copy that other warps add to concurrently: each count is read
// and cleared in one atomic exchange, so no concurrent increment is lost.
__device__ void warp_flush_shared(uint32_t *hw, int nb, unsigned long long *ghist, int lane)
{
    for (int b = 0; b < nb; ++b) {
        const u64 v = warp_sum_u64(atomicExch(&hw[b * 32 + lane], 0u));
        if (lane == 0 && v)
            atomicAdd(&ghist[b], v);
    }
}

// Candidate (column a, stencil offset) -> column pair, image, pruning
// (Sec. 2.2) and z reach, in binary64.  Returns false if the pair has no work.
__device__ __forceinline__ bool plan_item(const PairParams &P, int item, WorkItem &w)
{
    const int a = item / P.nstencil, s = item - a * P.nstencil;
    const int2 o = P.stencil[s];
    const int ax = a / P.g.ncy, ay = a - ax * P.g.ncy;
    int bx = ax + o.x, by = ay + o.y;
    int qx = 0, qy = 0;
    if (P.g.periodic) {
        qx = floor_div(bx, P.g.ncx);
        qy = floor_div(by, P.g.ncy);
        // an image two or more boxes away holds no pair within Rmax < L/2 (every
        // coordinate difference is below L), even when pruning is switched off
        if (qx < -1 || qx > 1 || qy < -1 || qy > 1)
            return false;
        bx -= qx * P.g.ncx;
        by -= qy * P.g.ncy;
    } else if (bx < 0 || bx >= P.g.ncx || by < 0 || by >= P.g.ncy) {
        return false;
    }
    const double Sx = qx * P.g.box[0], Sy = qy * P.g.box[1];
    const int b = bx * P.g.ncy + by;
    const long long nz = P.g.nz;
    if (P.shard_n > 1) {  // deterministic split of the primary columns over shards
        const unsigned long long total = P.A.cell_start[(long long)P.g.ncols * nz];
        const unsigned long long first = P.A.cell_start[a * nz];
        const unsigned long long lo = total * (unsigned long long)P.shard_k / P.shard_n;
        const unsigned long long hi = total * (unsigned long long)(P.shard_k + 1) / P.shard_n;
        if (first < lo || first >= hi)
            return false;
    }
    w.a0 = (int)P.A.cell_start[a * nz];
    w.a1 = (int)P.A.cell_start[(a + 1) * nz];
    w.b0 = (int)P.B.cell_start[b * nz];
    w.b1 = (int)P.B.cell_start[(b + 1) * nz];
    if (w.a0 >= w.a1 || w.b0 >= w.b1)
        return false;
    // minimum possible (x, y) separation of the two columns' bounding boxes
    const double4_32a ba = P.A.colbox[a], bb = P.B.colbox[b];
    const double gx = fmax(0.0, fmax(__dsub_rn(__dadd_rn(bb.x, Sx), ba.y),
                                     __dsub_rn(ba.x, __dadd_rn(bb.y, Sx))));
    const double gy = fmax(0.0, fmax(__dsub_rn(__dadd_rn(bb.z, Sy), ba.w),
                                     __dsub_rn(ba.z, __dadd_rn(bb.w, Sy))));
    const double g2 = __dadd_rn(__dmul_rn(gx, gx), __dmul_rn(gy, gy));
    if (!(P.flags & CF_FLAG_NO_PRUNE) && g2 >= P.prune_r2)
        return false;
    // z reach: dz_max,all of Sec. 2.2 (xi); pimax (rp-pi)
    double dzmax = P.rz;
    if (P.kind == 0)
        dzmax = sqrt(fmax(0.0, __dsub_rn(P.rxy2, __dmul_rn(g2, 1.0 - 1e-12))));
    w.dzmax = __dmul_rn(dzmax, 1.0 + 1e-9);
    const bool self = P.autocorr && o.x == 0 && o.y == 0;
    w.code = (qx + 1) | ((qy + 1) << 2) | (self ? 16 : 0) | (b << 5);
    w.wbase = 0;
    return true;
}

// Work-list kernel (a3): one thread per candidate, kept pairs appended to
// P.work with one warp-aggregated atomic per warp.  With the window pre-pass
// (P.win_chunk > 0) each kept pair also gets a run of window records,
// one per chunk of column a, from a second warp-aggregated counter.
__device__ __forceinline__ void worklist_body(const PairParams &P, int item)
{
    WorkItem w;
    const bool keep = item < P.n_items && plan_item(P, item, w);
    const unsigned m = __ballot_sync(FULL, keep);
    if (!m)
        return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    const int ch = P.win_chunk;
    unsigned nch = (keep && ch > 0) ? (unsigned)((w.a1 - w.a0 + ch - 1) / ch) : 0u;
    unsigned pre = nch;  // inclusive scan of the records over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(FULL, pre, o);
        if (lane >= o)
            pre += t;
    }
    const unsigned tot = __shfl_sync(FULL, pre, 31);
    unsigned base = 0, zb = 0;
    if (lane == leader) {
        base = atomicAdd(P.work_count, (unsigned)__popc(m));
        if (tot)
            zb = atomicAdd(P.win_count, tot);
    }
    base = __shfl_sync(FULL, base, leader);
    zb = __shfl_sync(FULL, zb, leader);
    if (keep) {
        if (ch > 0) {
            const long long first = (long long)zb + (long long)(pre - nch);
            if (first + (long long)nch > P.win_cap) {  // never with the host's bound
                atomicOr(P.err, ERR_INTERNAL);
                w.wbase = -1;
            } else {
                w.wbase = (int)first;
            }
        }
        P.work[base + __popc(m & ((1u << lane) - 1u))] = w;
    }
}

__global__ void __launch_bounds__(256) k_worklist(const __grid_constant__ PairParams P)
{
    worklist_body(P, blockIdx.x * blockDim.x + threadIdx.x);
}

// The work lists of every job of a batch in one launch: job j owns blocks
// [pre[j], pre[j + 1]) (one thread per candidate, as k_worklist).
__global__ void __launch_bounds__(256) k_worklist_batch(const PairParams *__restrict__ jobs,
                                                        const unsigned *__restrict__ pre, int njobs)
{
    __shared__ int s_job;
    if (threadIdx.x == 0) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pre[mid] <= blockIdx.x)
                lo = mid;
            else
                hi = mid - 1;
        }
        s_job = lo;
    }
    __syncthreads();
    const int j = s_job;
    worklist_body(jobs[j], (int)(blockIdx.x - pre[j]) * blockDim.x + threadIdx.x);
}

// One kept column pair, as the pair kernels use it (identical in every thread
// of the CTA: all read the same record).
struct Item {
    int a0, a1, b0, b1;
    double Sx, Sy, dzmax;
    bool self;
    int kmin, kmax;
    int wbase;  // first window record (window pre-pass); -1: none (error flagged)
};

// Per-CTA state a pair path carries from one work item to the next.
struct PathState {
    u64 n_eval, n_rck, n_viol;  // diagnostics (evaluations, re-checks, band violations)
    unsigned pending;           // pairs added to the shared u32 counts since the last flush
    unsigned phase;             // parity of the tile mbarrier
    unsigned wpend;             // weighted sums: pair slots per lane since the last row flush
};

__device__ __forceinline__ void decode_record(const PairParams &P, const WorkItem &w, Item &it)
{
    it.a0 = w.a0;
    it.a1 = w.a1;
    it.b0 = w.b0;
    it.b1 = w.b1;
    it.dzmax = w.dzmax;
    it.Sx = (double)((w.code & 3) - 1) * P.g.box[0];
    it.Sy = (double)(((w.code >> 2) & 3) - 1) * P.g.box[1];
    it.self = (w.code & 16) != 0;
    it.kmin = P.g.periodic ? (it.self ? 0 : -1) : 0;
    it.kmax = P.g.periodic ? 1 : 0;
    it.wbase = w.wbase;
}

__device__ __forceinline__ void decode_item(const PairParams &P, int item, Item &it)
{
    const WorkItem w = P.work[item];
    decode_record(P, w, it);
}

// First index p in [b0, b1) of column b with !(z[p] < v) (upper = false) or
// !(z[p] <= v) (upper = true); b1 if none.  The column is sorted by z (NaN
// padding at its end compares as larger than every value) and split into nz
// z-cells by the gridding's monotone rule cell_index_f: points of the cells
// below v's cell are < v and points of the cells above are > v, so the answer
// lies in v's cell and only that cell is searched.
__device__ __forceinline__ int zbound_col(const float *__restrict__ z, const uint32_t *__restrict__ cs,
                                          int nz, float inv_wz, int b0, int b1, float v, bool upper)
{
    const int c = cell_index_f(v, inv_wz, nz);
    int lo = max((int)cs[c], b0), hi = min((int)cs[c + 1], b1);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const float t = z[mid];
        if (upper ? (t <= v) : (t < v))
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Window pre-pass (Sec. 2.2, late entry and early exit on the sorted axis,
// applied per chunk of primaries): for every kept column pair (one warp) and
// every chunk of P.win_chunk z-consecutive points of column a (one lane), the
// ranges of column b whose z lies within the pair's reach dz of the chunk's z
// range, [z_lo - dz, z_hi + dz], per periodic z image, with the float32
// operations the pair kernel's own search would use.  The pair kernel then
// reads one record per chunk instead of searching its staged tile.
__global__ void __launch_bounds__(128) k_windows(const __grid_constant__ PairParams P)
{
    const int n_work = (int)*P.work_count;
    const int CH = P.win_chunk, lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int nz = P.g.nz;
    const float inv_wz = P.g.inv_wf[2];
    for (int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < n_work; item += nw) {
        const WorkItem w = P.work[item];
        if (w.wbase < 0)
            continue;
        Item it;
        decode_record(P, w, it);
        const uint32_t *cs = P.B.cell_start + (long long)(w.code >> 5) * nz;
        const float dzw = __fadd_ru(__double2float_ru(it.dzmax), P.zslack);
        const float zb_lo = P.B.zs[it.b0];  // column b's z range (a window outside it is empty)
        float zb_hi = P.B.zs[it.b1 - 1];
        if (isnan(zb_hi))
            zb_hi = INFINITY;
        const int nch = (it.a1 - it.a0 + CH - 1) / CH;
        for (int c = lane; c < nch; c += 32) {
            const int ib = it.a0 + c * CH;
            int ie = min(ib + CH, it.a1) - 1;
            const float zlo = P.A.zs[ib];
            float zhi = P.A.zs[ie];
            while (ie > ib && isnan(zhi))  // column padding: the largest real z is earlier
                zhi = P.A.zs[--ie];
            Win wn;
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) {
                const int k = kk - 1;
                int lo = 0, hi = 0;
                if (!isnan(zlo) && k >= it.kmin && k <= it.kmax) {
                    const float kz = (float)k * P.boxf[2];
                    const float wlo = zlo - kz - dzw, whi = zhi - kz + dzw;
                    if (!(whi < zb_lo || wlo > zb_hi)) {
                        lo = zbound_col(P.B.zs, cs, nz, inv_wz, it.b0, it.b1, wlo, false);
                        hi = zbound_col(P.B.zs, cs, nz, inv_wz, lo, it.b1, whi, true);
                    }
                }
                wn.lo[kk] = lo;
                wn.hi[kk] = hi;
            }
            P.win[w.wbase + c] = wn;
        }
    }
}

// Byte offset in the shared block of the chunk counter that the warps of a CTA
// claim chunks of the staged tile from ([0, 128) holds the barrier, the item).
constexpr int CLAIM_OFF = 16;

// Stage the float32 x, y, z tiles (three 1-D bulk copies, one mbarrier):
// thread 0 issues the copies, every thread pads and waits (bounded).  The
// source slices start at a multiple of 4 floats and hold a multiple of 4 (the
// gridded columns are padded), as the bulk copy requires.  False in every
// thread if the wait gave up.
__device__ __forceinline__ bool stage_tiles32(unsigned char *smem, const Gridded &B, int t0,
                                              int count, uint64_t *bar, unsigned &phase,
                                              unsigned *err, uint64_t wait_ns, bool with_w = false)
{
    __syncthreads();  // previous tile fully consumed
    const unsigned bytes = (unsigned)count * 4u;
    if (threadIdx.x == 0) {
        *reinterpret_cast<volatile int *>(smem + CLAIM_OFF) = 0;  // chunk counter of the new tile
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, (with_w ? 4u : 3u) * bytes);
        bulk_g2s(smem + XI32_TX_OFF, B.xs + t0, bytes, bar);
        bulk_g2s(smem + XI32_TX_OFF + XI32_TSTRIDE, B.ys + t0, bytes, bar);
        bulk_g2s(smem + XI32_TX_OFF + 2 * XI32_TSTRIDE, B.zs + t0, bytes, bar);
        if (with_w)
            bulk_g2s(smem + XIW_W_OFF, B.ws + t0, bytes, bar);
    }
    float *t = reinterpret_cast<float *>(smem + XI32_TX_OFF);
    for (int s = threadIdx.x; s < 3 * 64; s += THREADS)  // sentinels: never counted
        t[(s >> 6) * (XI32_TSTRIDE / 4) + count + (s & 63)] = __int_as_float(0x7fc00000);
    if (with_w)
        for (int s = threadIdx.x; s < 64; s += THREADS)
            reinterpret_cast<float *>(smem + XIW_W_OFF)[count + s] = 0.0f;
    const bool ok = mbar_wait(bar, phase, wait_ns);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            atomicOr(err, ERR_TIMEOUT);
            mbar_wait(bar, phase, wait_ns);  // a copy still in flight lands before the CTA exits
        }
        __syncthreads();
        phase ^= 1u;
        return false;
    }
    phase ^= 1u;
    return true;
}

// Issue the bulk copy of one tile (thread 0), pad, wait (all threads, bounded).
// Returns false (in every thread) if the wait gave up.
template <class T>
__device__ __forceinline__ bool stage_tile(T *tile, const T *src, int count, int pad_elems,
                                           uint64_t *bar, unsigned &phase, unsigned *err,
                                           uint64_t wait_ns)
{
    __syncthreads();  // previous tile fully consumed
    if (threadIdx.x == 0) {
        *reinterpret_cast<volatile int *>(reinterpret_cast<unsigned char *>(bar) + CLAIM_OFF) = 0;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, (unsigned)(count * sizeof(T)));
        bulk_g2s(tile, src, (unsigned)(count * sizeof(T)), bar);
    }
    for (int s = threadIdx.x; s < pad_elems; s += THREADS) {
        T nanv;
        const float q = __int_as_float(0x7fc00000);
        nanv.x = nanv.y = nanv.z = nanv.w = q;
        tile[count + s] = nanv;  // sentinels after the copied range: never counted
    }
    const bool ok = mbar_wait(bar, phase, wait_ns);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            atomicOr(err, ERR_TIMEOUT);
            mbar_wait(bar, phase, wait_ns);  // a copy still in flight lands before the CTA exits
        }
        __syncthreads();
        phase ^= 1u;
        return false;
    }
    phase ^= 1u;
    return true;
}

// ============================================================ float32 kernel
// Shared layout of the float32 DD(r) kernels (compile-time offsets, so table
// and tile addresses fold into load immediates): [0,128) barrier + item; LUT
// (LUT_MAX bytes); x, y, z tiles of TILE32 + 64 floats; thresholds; squared
// edges; histogram copies (the pipelined kernel's second tile buffer follows).
constexpr int LUT_OFF = XI32_LUT_OFF;
constexpr int TX_OFF = XI32_TX_OFF;
constexpr int TSTRIDE = XI32_TSTRIDE;
constexpr int THR_OFF = XI32_THR_OFF;
constexpr int E2_OFF = XI32_E2_OFF;
constexpr int HIST_OFF = XI32_HIST_OFF;

// Per-window constants of the sweep.
struct Sweep32 {
    const unsigned char *tb;  // staged tile: x, y, z arrays TSTRIDE bytes apart
    int t0;                   // global index of tile element 0
    int nb;                   // bins; row nb is the dummy row
    uint32_t u0, lut_last;
    int shift;
    int nthr;
    int lin;                  // table cells linear in d2 (scale lscale) or logarithmic
    float lscale;
    const double4_32a *pa, *pb;
    double Sx, Sy, Sz;
};

__device__ __forceinline__ uint32_t lut_byte(const unsigned char *smem, uint32_t u0s, int shift,
                                             uint32_t last, float d2)
{
    const uint32_t q = (__float_as_uint(d2) >> shift) - u0s;  // below-range values wrap to huge
    return smem[LUT_OFF + min(q, last)];
}

// Cells linear in d2: adding 2^23 in the fma rounds d2 * scale to an integer q
// held in the sum's low bits (exact below 2^22; larger values, and NaN, give
// larger bit patterns and clamp to the out-of-range entry).
constexpr float LIN_MAGIC = 8388608.0f;  // 2^23: spacing 1 in [2^23, 2^24)
constexpr uint32_t LIN_MAGIC_BITS = 0x4b000000u;

__device__ __forceinline__ uint32_t lut_byte_lin(const unsigned char *smem, float scale,
                                                 uint32_t last, float d2)
{
    const uint32_t q = __float_as_uint(__fmaf_rn(d2, scale, LIN_MAGIC)) - LIN_MAGIC_BITS;
    return smem[LUT_OFF + min(q, last)];
}

template <bool LIN>
__device__ __forceinline__ uint32_t lut_entry(const unsigned char *smem, uint32_t u0s, int shift,
                                              uint32_t last, float scale, float d2)
{
    return LIN ? lut_byte_lin(smem, scale, last, d2) : lut_byte(smem, u0s, shift, last, d2);
}

// Number of thresholds T[c] <= d2 (T non-decreasing, d2 not NaN), scanning
// down from the top: flagged cells are dominated by the largest edges (the
// pair density grows with the separation), where this ends in a step or two.
__device__ __forceinline__ int thr_count_top(const float *T, int nthr, float d2)
{
    int c = nthr;
    while (c > 0 && T[c - 1] > d2)
        --c;
    return c;
}

// Number of thresholds T[c] <= d2 (T is non-decreasing; NaN counts none).
__device__ __forceinline__ int thr_count(const float *T, int nthr, float d2)
{
    int lo = 0, hi = nthr;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (T[mid] <= d2)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void red_shared1(uint32_t addr)
{
    asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(addr));
}

// Table byte at a shared address, sign-extended: the flagged entry gives -1.
__device__ __forceinline__ uint32_t lds_entry(uint32_t addr)
{
    uint32_t e;
    asm volatile("ld.shared.s8 %0, [%1];" : "=r"(e) : "r"(addr));
    return e;
}

// (m << 1) | (v >> 31): one funnel shift appends v's sign bit to the mask m.
__device__ __forceinline__ uint32_t push_sign(uint32_t m, uint32_t v)
{
    uint32_t r;
    asm("shf.l.wrap.b32 %0, %1, %2, 1;" : "=r"(r) : "r"(v), "r"(m));
    return r;
}

// Flagged table cell: count the thresholds <= d2; inside a band re-evaluate in
// binary64.  Adds the pair to its true bin (the main path has already put it in
// the flagged row, which is never read).  Returns 1 if re-evaluated.
__device__ __forceinline__ int resolve_pair(const unsigned char *smem, const Sweep32 &S,
                                            uint32_t hl, float d2, int i, int jg)
{
    const float *T = reinterpret_cast<const float *>(smem + THR_OFF);
    const int c = thr_count_top(T, S.nthr, d2);
    int row;
    int re = 0;
    if (!(c & 1)) {
        row = (c >= 2 && c <= 2 * S.nb) ? (c - 2) >> 1 : -1;
    } else {
        row = recheck64(reinterpret_cast<const double *>(smem + E2_OFF), S.nb, S.pa, S.pb, i, jg,
                        S.Sx, S.Sy, S.Sz);
        re = 1;
    }
    if (row >= 0)
        red_shared1(hl + (uint32_t)row * 128u);
    return re;
}

// ---- weighted sums in the float32 DD(r) sweep (Code 1's weight per pair)
// A pair adds round(v * scale) for its weight v = w_i w_j (scale sw) and for
// r * v (a scale per bin) to 32-bit per-lane rows, as the low mantissa bits of
// fma(v, scale, 1.5 * 2^23): the row then holds count * bits(1.5 * 2^23) plus
// the exact integer sum, which the lane recovers with its own count.  Scales
// are powers of two with every term below 2^21 in size, so 512 terms cannot
// overflow; rows move to per-thread 64-bit sums every 64 iterations.  The
// rounding error of one term is at most half a unit: relative to the term
// 2^-22 max|w_i w_j| / |w_i w_j| (times Rmax / e_k for r w).
constexpr float QMAGIC = 12582912.0f;      // 1.5 * 2^23
constexpr uint32_t QMAGIC_BITS = 0x4b400000u;
constexpr unsigned WFLUSH_PAIRS = 448;     // flush before any row holds more terms

struct WAcc {
    uint32_t hlw, hlr;     // shared addresses of this lane's w and r w rows (row stride 128 B)
    const float *sr;       // per-row scale of r w (shared; 0 for the two dummy rows)
    float sw;              // scale of w
    const float *wsj;      // secondary weights of the staged tile (global, from tile element 0)
    const float *xlj, *ylj, *zlj;  // secondaries' coordinate residuals (global, from tile element 0)
    uint32_t *cnt, *wq, *rq;  // this lane's rows (generic pointers, stride 32 words)
    long long *g;          // this thread's [bin][count, w, r w] 64-bit sums (global)
    int nb;
};

__device__ __forceinline__ void red_shared_u32(uint32_t addr, uint32_t v)
{
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}

template <bool W, bool RV>
__device__ __forceinline__ void wacc_add(const WAcc &A, uint32_t e, float pw, float d2)
{
    if (W)
        red_shared_u32(A.hlw + e * 128u, __float_as_uint(__fmaf_rn(pw, A.sw, QMAGIC)));
    if (RV) {
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d2));
        const float rw = W ? r * pw : r;
        red_shared_u32(A.hlr + e * 128u, __float_as_uint(__fmaf_rn(rw, A.sr[(int)e], QMAGIC)));
    }
}

// Move this lane's rows of the counted bins to its 64-bit sums (lane-private).
template <bool W, bool RV>
__device__ __noinline__ void wacc_flush(const WAcc &A)
{
    for (int k = 0; k < A.nb; ++k) {
        const uint32_t c = A.cnt[k * 32];
        if (!c)
            continue;
        A.cnt[k * 32] = 0u;
        A.g[3 * k] += (long long)c;
        if (W) {
            A.g[3 * k + 1] += (long long)(int)(A.wq[k * 32] - c * QMAGIC_BITS);
            A.wq[k * 32] = 0u;
        }
        if (RV) {
            A.g[3 * k + 2] += (long long)(int)(A.rq[k * 32] - c * QMAGIC_BITS);
            A.rq[k * 32] = 0u;
        }
    }
}

// A flagged pair recorded by sweep32: recompute its float32 d2 from the
// staged tile (the same IEEE operations as the packed main path), settle it
// with the thresholds (binary64 inside a band) and add it to its true row.
template <bool W, bool RV, bool RL = false>
__device__ __forceinline__ int resolve_local(const unsigned char *smem, const Sweep32 &S, uint32_t hl,
                                          float xh, float yh, float zh, int i, int jl,
                                          const WAcc &A, float wi, float lx = 0.0f, float ly = 0.0f,
                                          float lz = 0.0f)
{
    const float *tx = reinterpret_cast<const float *>(S.tb);
    const float dx = __fsub_rn(tx[jl], xh);
    const float dy = __fsub_rn(tx[jl + TSTRIDE / 4], yh);
    const float dz = __fsub_rn(tx[jl + TSTRIDE / 2], zh);
    const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    // the mean separation's squared distance with the coordinates' residuals
    const float dc = RL ? __fmaf_rn(2.0f, __fmaf_rn(dz, A.zlj[jl] - lz, __fmaf_rn(dy, A.ylj[jl] - ly,
                                                                                 dx * (A.xlj[jl] - lx))),
                                    d2)
                        : d2;
    if (!W && !RV)
        return resolve_pair(smem, S, hl, d2, i, S.t0 + jl);
    const float *T = reinterpret_cast<const float *>(smem + THR_OFF);
    const int c = thr_count_top(T, S.nthr, d2);
    int row, re = 0;
    if (!(c & 1)) {
        row = (c >= 2 && c <= 2 * S.nb) ? (c - 2) >> 1 : -1;
    } else {
        row = recheck64(reinterpret_cast<const double *>(smem + E2_OFF), S.nb, S.pa, S.pb, i,
                        S.t0 + jl, S.Sx, S.Sy, S.Sz);
        re = 1;
    }
    if (row >= 0) {
        red_shared1(hl + (uint32_t)row * 128u);
        wacc_add<W, RV>(A, (uint32_t)row, W ? __fmul_rn(A.wsj[jl], wi) : 1.0f, dc);
    }
    return re;
}

// 8-byte shared load at a 32-bit shared address plus a constant offset.
template <int OFF>
__device__ __forceinline__ u64 lds64(uint32_t a)
{
    u64 v;
    asm volatile("ld.shared.b64 %0, [%1+%2];" : "=l"(v) : "r"(a), "n"(OFF));
    return v;
}

// 16-byte shared load (four floats as two packed pairs) at a 32-bit shared
// address plus a constant offset.
template <int OFF>
__device__ __forceinline__ void lds128(uint32_t a, u64 &lo, u64 &hi)
{
    asm volatile("ld.shared.v2.b64 {%0, %1}, [%2+%3];" : "=l"(lo), "=l"(hi) : "r"(a), "n"(OFF));
}

// Sweep one window [jlo, jhi) of the staged tile.  Lane (ii, jj) holds PP
// primaries (each broadcast to both halves of packed registers) and evaluates
// them against four consecutive secondaries j .. j+3 (one 16-byte shared load
// per axis feeds 4 PP pairs); a step covers I PP primaries x 128 / I
// secondaries.  Pairs whose table cell is flagged go to the flagged row and set
// a bit of the lane's mask; once per block of 8 steps a warp-uniform test
// settles the recorded pairs (so the loop body has no data-dependent branch).
// RL: the mean separation's r comes from the squared distance corrected with
// the coordinates' float32 rounding residuals (secondaries' from the residual
// tiles, primaries' in LX, LY, LZ, shift roundings included):
// d2 = d2~ + 2 (dx~ ex + dy~ ey + dz~ ez) up to the square of the residuals.
template <int I, int PP, bool TRI, bool EVALS, bool VERIFY, bool LIN, bool W, bool RV, bool RL = false>
__device__ __forceinline__ void sweep32(unsigned char *smem, const Sweep32 &S, uint32_t hl, int jlo,
                                        int jhi, int jj, const u64 (&XH)[PP], const u64 (&YH)[PP],
                                        const u64 (&ZH)[PP], const int (&iv)[PP],
                                        const bool (&vv)[PP], u64 &n_eval, u64 &n_rck, u64 &n_viol,
                                        const WAcc &A, const float (&wi)[PP], unsigned &wpend,
                                        u64 LX, u64 LY, u64 LZ)
{
    static_assert(!RL || PP == 1, "residual-corrected separations take one primary per lane");
    const u64 TWO = pack2(2.0f, 2.0f);
    const float qnan = __int_as_float(0x7fc00000);
    const int jstart = jlo & ~3;  // 16-byte aligned quads; extra j's are never counted
    constexpr int JS = 128 / I;   // secondaries per step (four per lane group)
    const int nit = (jhi - jstart + JS - 1) / JS;
    const u64 LS = pack2(S.lscale, S.lscale), LM = pack2(LIN_MAGIC, LIN_MAGIC);
    // shared addresses of the table: fma(d2, s, 2^23) >= 2^23 (d2 >= 0, NaN larger),
    // so bits - LIN_MAGIC_BITS never wraps and the base folds into the clamp
    const uint32_t lutb = smem_u32(smem + LUT_OFF), lut_lo = lutb - LIN_MAGIC_BITS,
                   lut_hi = lutb + S.lut_last;
    for (int b0 = 0; b0 < nit; b0 += 8) {
        const int jAb = jstart + 4 * jj + b0 * JS;
        const uint32_t pb = smem_u32(S.tb) + jAb * 4;
        const int tend = min(8, nit - b0);
        uint32_t fm[PP];
#pragma unroll
        for (int q = 0; q < PP; ++q)
            fm[q] = 0u;
        for (int t = 0; t < tend; ++t) {
            const uint32_t p = pb + t * 4 * JS;
            const int jA = jAb + t * JS;
            u64 xA, xB, yA, yB, zA, zB;  // (j, j+1) and (j+2, j+3)
            lds128<0>(p, xA, xB);
            lds128<TSTRIDE>(p, yA, yB);
            lds128<2 * TSTRIDE>(p, zA, zB);
            float d[PP][4];
            float dr[PP][4];     // residual-corrected squared separations (RL only)
            float pw[PP][4];     // pair weights (weighted sums only)
            uint32_t cq[PP][4];  // table cell of each pair
            u64 lxA = 0, lxB = 0, lyA = 0, lyB = 0, lzA = 0, lzB = 0;
            if (RL) {  // residuals of the four secondaries (global, 16-byte aligned)
                const float4 rx = *reinterpret_cast<const float4 *>(A.xlj + jA);
                const float4 ry = *reinterpret_cast<const float4 *>(A.ylj + jA);
                const float4 rz = *reinterpret_cast<const float4 *>(A.zlj + jA);
                lxA = pack2(rx.x, rx.y);
                lxB = pack2(rx.z, rx.w);
                lyA = pack2(ry.x, ry.y);
                lyB = pack2(ry.z, ry.w);
                lzA = pack2(rz.x, rz.y);
                lzB = pack2(rz.z, rz.w);
            }
            if (W) {  // w_j of the four secondaries (global, 16-byte aligned)
                const float4 wv = *reinterpret_cast<const float4 *>(A.wsj + jA);
                const u64 wA = pack2(wv.x, wv.y), wB = pack2(wv.z, wv.w);
#pragma unroll
                for (int q = 0; q < PP; ++q) {
                    const u64 WI = pack2(wi[q], wi[q]);
                    unpack2(fmul2(wA, WI), pw[q][0], pw[q][1]);
                    unpack2(fmul2(wB, WI), pw[q][2], pw[q][3]);
                }
            }
#pragma unroll
            for (int q = 0; q < PP; ++q) {
                u64 dx = fsub2(xA, XH[q]), dy = fsub2(yA, YH[q]), dz = fsub2(zA, ZH[q]);
                const u64 dA = ffma2(dz, dz, ffma2(dy, dy, fmul2(dx, dx)));
                if (RL) {
                    const u64 c = ffma2(dz, fsub2(lzA, LZ), ffma2(dy, fsub2(lyA, LY), fmul2(dx, fsub2(lxA, LX))));
                    unpack2(ffma2(TWO, c, dA), dr[q][0], dr[q][1]);
                }
                dx = fsub2(xB, XH[q]);
                dy = fsub2(yB, YH[q]);
                dz = fsub2(zB, ZH[q]);
                const u64 dB = ffma2(dz, dz, ffma2(dy, dy, fmul2(dx, dx)));
                if (RL) {
                    const u64 c = ffma2(dz, fsub2(lzB, LZ), ffma2(dy, fsub2(lyB, LY), fmul2(dx, fsub2(lxB, LX))));
                    unpack2(ffma2(TWO, c, dB), dr[q][2], dr[q][3]);
                }
                unpack2(dA, d[q][0], d[q][1]);
                unpack2(dB, d[q][2], d[q][3]);
                if (LIN) {  // one packed fma gives two cells
                    float t[4];
                    unpack2(ffma2(dA, LS, LM), t[0], t[1]);
                    unpack2(ffma2(dB, LS, LM), t[2], t[3]);
#pragma unroll
                    for (int r = 0; r < 4; ++r)  // the table byte's shared address
                        cq[q][r] = min(__float_as_uint(t[r]) + lut_lo, lut_hi);
                } else {
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        cq[q][r] = lutb + min((__float_as_uint(d[q][r]) >> S.shift) - S.u0, S.lut_last);
                }
            }
            const int gA = S.t0 + jA;  // global index of secondary r is gA + r
            if (TRI) {  // pairs with j <= i: the out-of-range entry (and NaN for the checks)
#pragma unroll
                for (int q = 0; q < PP; ++q)
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        cq[q][r] = gA + r > iv[q] ? cq[q][r] : lut_hi;
                        d[q][r] = gA + r > iv[q] ? d[q][r] : qnan;
                    }
            }
            if (EVALS) {
#pragma unroll
                for (int q = 0; q < PP; ++q)
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        n_eval += (vv[q] && jA + r >= jlo && jA + r < jhi && (!TRI || gA + r > iv[q]))
                                      ? 1ull : 0ull;
            }
#pragma unroll
            for (int q = 0; q < PP; ++q) {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const uint32_t e = lds_entry(cq[q][r]);  // the row: bin, dummy or flagged (-1)
                    red_shared1(hl + e * 128u);
                    if (W || RV)
                        wacc_add<W, RV>(A, e, W ? pw[q][r] : 1.0f, RL ? dr[q][r] : d[q][r]);
                    // pair (t, r) ends at bit 4 tend - 1 - (4 t + r) of the mask
                    fm[q] = push_sign(fm[q], e);
                }
            }
            if (VERIFY) {
                const float *T = reinterpret_cast<const float *>(smem + THR_OFF);
                const double *E2 = reinterpret_cast<const double *>(smem + E2_OFF);
                // pairs with real points on both sides (sentinels and padding give NaN)
#pragma unroll
                for (int q = 0; q < PP; ++q)
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (vv[q] && !isnan(d[q][r]))
                            n_viol += verify_pair(d[q][r], T, S.nthr, S.nb, E2, S.pa, S.pb, iv[q],
                                                  gA + r, S.Sx, S.Sy, S.Sz);
            }
        }
        uint32_t anyf = 0u;
#pragma unroll
        for (int q = 0; q < PP; ++q)
            anyf |= fm[q];
        if (__any_sync(FULL, anyf != 0u)) {
#pragma unroll
            for (int q = 0; q < PP; ++q) {
                float xh, yh, zh, lx = 0.0f, ly = 0.0f, lz = 0.0f, tmp;
                unpack2(XH[q], xh, tmp);
                unpack2(YH[q], yh, tmp);
                unpack2(ZH[q], zh, tmp);
                if (RL) {
                    unpack2(LX, lx, tmp);
                    unpack2(LY, ly, tmp);
                    unpack2(LZ, lz, tmp);
                }
                uint32_t m = fm[q];
                while (m) {
                    const int bit = __ffs(m) - 1;
                    m &= m - 1u;
                    const int k = 4 * tend - 1 - bit;  // = 4 t + r
                    const int jl = jAb + (k >> 2) * JS + (k & 3);
                    n_rck += resolve_local<W, RV, RL>(smem, S, hl, xh, yh, zh, iv[q], jl, A, wi[q],
                                                      lx, ly, lz);
                }
            }
        }
        if (W || RV) {  // warp-uniform: every lane ran the same iterations
            wpend += (unsigned)tend * 4u * PP;
            if (wpend > WFLUSH_PAIRS - 64u * PP) {
                wacc_flush<W, RV>(A);
                wpend = 0;
            }
        }
    }
}

// Lane-parallel search for the first index in [start, n) whose key is >= v
// (upper = false) or > v (upper = true), assuming it is at least start: one
// probe round at stride 4 from start, then a short or general search.
template <class Key, class V>
__device__ __forceinline__ int warp_bound_from(Key key, int start, int n, V v, bool upper, int lane)
{
    const int p = start + 4 * lane;
    bool q = false;
    if (p < n) {
        const V z = key(p);
        q = upper ? (z <= v) : (z < v);
    }
    const int c = __popc(__ballot_sync(FULL, q));
    if (c == 0)
        return start;
    const int lo = start + 4 * (c - 1) + 1;
    const int hi = c < 32 ? min(n, start + 4 * c) : n;
    return lo + warp_bound([&](int t) { return key(lo + t); }, hi - lo, v, upper, lane);
}

// Weighted float32 DD(r): shared rows after the count rows, [warp][row][lane]
// for w, then for r w, then the per-row scale of r w; power-of-two scales from
// the largest weights (gridding wrote their bit patterns).
__device__ __forceinline__ float pow2_floor(float x)
{
    return (x > 0.0f && x < INFINITY) ? __uint_as_float(__float_as_uint(x) & 0x7f800000u) : 1.0f;
}

__device__ __forceinline__ float wmax_pair(const PairParams &P)
{
    return __uint_as_float(*P.A.wmax) * __uint_as_float(*P.B.wmax);
}

// Rounding error of s = fl(a + b), i.e. a + b - s exactly (Knuth's TwoSum).
__device__ __forceinline__ float two_sum_err(float a, float b, float s)
{
    const float bb = __fsub_rn(s, a);
    return __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// HC histogram copies, each shared by WARPS / HC warps (red.shared is atomic);
// the weighted rows are per warp.  PREWIN: chunk windows come from the window
// pre-pass (k_windows) instead of searches of the staged tile.  LT: table
// cells linear in d2 (1), on float bits (0), or as the launch's tables say (-1).
// RL: mean separations from residual-corrected squared distances (sweep32).
template <int I, int PP, bool EVALS, bool VERIFY, bool W = false, bool RV = false, int HC = WARPS,
          bool PREWIN = false, int LT = -1, bool RL = false>
struct Xi32Path {
    static_assert(HC == WARPS || !(W || RV), "weighted rows are per warp");
    static_assert(WARPS % HC == 0, "warps share copies evenly");

    static __device__ __forceinline__ void init(const PairParams &P, unsigned char *smem)
    {
        // I * PP primaries per chunk (lane ii = lane % I holds primaries ii, ii + I,
        // ...); jj = lane / I picks the pair of secondaries.
        const int nb = P.nbins;
        float *thr = reinterpret_cast<float *>(smem + THR_OFF);
        double *E2 = reinterpret_cast<double *>(smem + E2_OFF);
        uint32_t *hist = reinterpret_cast<uint32_t *>(smem + HIST_OFF);

        const int tid = threadIdx.x;
        for (int q = tid; q < P.lut_n; q += THREADS)
            smem[LUT_OFF + q] = P.lut[q];
        for (int q = tid; q < P.nthr; q += THREADS)
            thr[q] = P.thr[q];
        for (int q = tid; q <= nb; q += THREADS)
            E2[q] = P.E2[q];
        constexpr int planes = 1 + (W ? 1 : 0) + (RV ? 1 : 0);
        for (int q = tid; q < planes * HC * (nb + 2) * 32; q += THREADS)
            hist[q] = 0u;
        if (W || RV) {
            float *sr = reinterpret_cast<float *>(hist + planes * WARPS * (nb + 2) * 32);
            const float mw = W ? wmax_pair(P) : 1.0f;
            for (int k = tid; k < nb + 2; k += THREADS)  // r w < 2^20 scale in bin k - 1 (headroom 2)
                sr[k] = (k >= 1 && k <= nb) ? pow2_floor(1048576.0f / (sqrtf((float)E2[k]) * mw)) : 0.0f;
            long long *g = P.wscratch + ((long long)blockIdx.x * THREADS + tid) * 3 * nb;
            for (int k = 0; k < 3 * nb; ++k)
                g[k] = 0;
        }
    }

    // One work item through the CTA's single tile buffer: stage each tile of
    // column b, then sweep it.
    static __device__ __forceinline__ bool item(const PairParams &P, const Item &it,
                                                unsigned char *smem, PathState &st)
    {
        uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
        for (int t0 = it.b0; t0 < it.b1; t0 += TILE32) {
            const int nt = min(TILE32, it.b1 - t0);
            if (!stage_tiles32(smem, P.B, t0, nt, bar, st.phase, P.err, P.wait_ns))
                return false;
            tile(P, it, t0, nt, smem + TX_OFF, reinterpret_cast<int *>(smem + CLAIM_OFF), smem, st);
        }
        return true;
    }

    // Sweep the staged tile [t0, t0 + nt) of column b (at tb) against every
    // chunk of column a; the warps claim chunks from *claim in increasing order.
    static __device__ __forceinline__ void tile(const PairParams &P, const Item &it, int t0, int nt,
                                                const unsigned char *tb, int *claim,
                                                unsigned char *smem, PathState &st)
    {
        // I * PP primaries per chunk (lane ii = lane % I holds primaries ii, ii + I,
        // ...); jj = lane / I picks the pair of secondaries.
        constexpr int CH = I * PP;
        const int nb = P.nbins;
        const float *tz = reinterpret_cast<const float *>(tb + 2 * TSTRIDE);
        uint32_t *hist = reinterpret_cast<uint32_t *>(smem + HIST_OFF);

        const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
        u64 &n_eval = st.n_eval;
        u64 &n_rck = st.n_rck;
        u64 &n_viol = st.n_viol;
        unsigned &pending = st.pending;

        // row 0 of the warp's copy (rows: flagged at -1, the bins, not counted)
        uint32_t *hw = hist + ((warp % HC) * (nb + 2) + 1) * 32;
        const uint32_t hl = smem_u32(hw + lane);  // this lane's histogram column (shared address)
        const int ii = lane % I, jj = lane / I;
        WAcc A;
        if (W || RV) {
            const int plane = WARPS * (nb + 2) * 32;
            A.cnt = hw + lane;
            A.wq = A.cnt + plane;
            A.rq = A.cnt + (W ? 2 : 1) * plane;
            A.hlw = smem_u32(A.wq);
            A.hlr = smem_u32(A.rq);
            A.sr = reinterpret_cast<const float *>(hist + (1 + (W ? 1 : 0) + (RV ? 1 : 0)) * plane) + 1;
            A.sw = W ? pow2_floor(2097152.0f / wmax_pair(P)) : 1.0f;
            A.wsj = P.B.ws;
            A.g = P.wscratch + ((long long)blockIdx.x * THREADS + tid) * 3 * nb;
            A.nb = nb;
        }
        Sweep32 S;
        S.nb = nb;
        S.u0 = P.u0;
        S.lut_last = (uint32_t)(P.lut_n - 1);
        S.shift = P.lut_shift;
        S.nthr = P.nthr;
        S.lin = P.lut_lin;
        S.lscale = P.lut_scale;
        S.pa = P.A.pos64;
        S.pb = P.B.pos64;
        const float qnan = __int_as_float(0x7fc00000);

        // Chunk windows (late entry / early exit per chunk, Sec. 2.2): the chunk's
        // z range widened by the column pair's reach, per periodic z image;
        // with PREWIN read from the window pre-pass, else searched in the tile.
        const float dzw = __fadd_ru(__double2float_ru(it.dzmax), P.zslack);
        const float Sxf = __double2float_rn(it.Sx), Syf = __double2float_rn(it.Sy);
        // RL: the roundings of the periodic shifts, S - fl32(S) and L_z - fl32(L_z)
        const float dSx = RL ? __double2float_rn(__dsub_rn(it.Sx, (double)Sxf)) : 0.0f;
        const float dSy = RL ? __double2float_rn(__dsub_rn(it.Sy, (double)Syf)) : 0.0f;
        const float dLz = RL ? __double2float_rn(__dsub_rn(P.g.box[2], (double)P.boxf[2])) : 0.0f;
        if (RL) {
            A.xlj = P.B.xl + t0;
            A.ylj = P.B.yl + t0;
            A.zlj = P.B.zl + t0;
        }
        S.Sx = it.Sx;
        S.Sy = it.Sy;
        const int nchunks = (it.a1 - it.a0 + CH - 1) / CH;
        S.tb = tb;
        S.t0 = t0;
        if (PREWIN && it.wbase < 0)
            return;  // no window records (the work-list kernel flagged an error)
        const float zt_lo = tz[0];
        float zt_hi = tz[nt - 1];
        if (isnan(zt_hi))  // padding at the column end: largest real z is earlier
            zt_hi = INFINITY;
        auto zkey = [&](int q) { return tz[q]; };
        int lo_prev[3] = {0, 0, 0}, hi_prev[3] = {0, 0, 0};  // windows searched before
        auto next_chunk = [&]() {
            int v = 0;
            if (lane == 0)
                v = atomicAdd(claim, 1);
            return __shfl_sync(FULL, v, 0);
        };
        const bool lin = LT < 0 ? S.lin != 0 : LT == 1;
        for (int c = next_chunk(); c < nchunks; c = next_chunk()) {
            const int ib = it.a0 + c * CH;
            u64 XH[PP], YH[PP], ZH[PP];
            u64 LX = 0, LY = 0, LZ = 0;  // the primary's shifted residuals (RL, one primary per lane)
            int iv[PP];
            bool vv[PP];
            float zq[PP], wi[PP];
            float lzq = 0.0f;
            float zmax = qnan;
            int wl0 = 0, wl1 = 0, wl2 = 0, wh0 = 0, wh1 = 0, wh2 = 0;
            if (PREWIN) {  // this chunk's windows in column b (three 8-byte loads)
                const int2 *wr = reinterpret_cast<const int2 *>(P.win + it.wbase + c);
                const int2 r0 = wr[0], r1 = wr[1], r2 = wr[2];
                wl0 = r0.x;
                wl1 = r0.y;
                wl2 = r1.x;
                wh0 = r1.y;
                wh1 = r2.x;
                wh2 = r2.y;
            }
#pragma unroll
            for (int q = 0; q < PP; ++q) {
                const int i = ib + q * I + ii;
                float xi = qnan, yi = qnan, zi = qnan;
                wi[q] = 1.0f;
                if (i < it.a1) {
                    xi = P.A.xs[i];
                    yi = P.A.ys[i];
                    zi = P.A.zs[i];
                    if (W)
                        wi[q] = P.A.ws[i];
                }
                iv[q] = i;
                vv[q] = !isnan(xi);  // chunk tail and column padding are NaN
                const float xh = __fsub_rn(xi, Sxf), yh = __fsub_rn(yi, Syf);
                XH[q] = pack2(xh, xh);
                YH[q] = pack2(yh, yh);
                zq[q] = zi;
                if (RL) {  // the primary's residuals after the shift: r_i + (x~ - S~ - x^) - (S - S~)
                    float rx = 0.0f, ry = 0.0f;
                    if (i < it.a1) {
                        rx = P.A.xl[i];
                        ry = P.A.yl[i];
                        lzq = P.A.zl[i];
                    }
                    const float lx = __fsub_rn(__fadd_rn(rx, two_sum_err(xi, -Sxf, xh)), dSx);
                    const float ly = __fsub_rn(__fadd_rn(ry, two_sum_err(yi, -Syf, yh)), dSy);
                    LX = pack2(lx, lx);
                    LY = pack2(ly, ly);
                }
                if (!PREWIN)
                    zmax = (isnan(zmax) || zi > zmax) ? zi : zmax;
            }
            float zlo = 0.0f, zhi = 0.0f;
            if (!PREWIN) {
                zlo = __shfl_sync(FULL, zq[0], 0);
                zhi = zmax;
#pragma unroll
                for (int o = 1; o < I; o <<= 1) {  // largest real z of the chunk
                    const float t = __shfl_xor_sync(FULL, zhi, o);
                    zhi = (isnan(zhi) || t > zhi) ? t : zhi;
                }
                if (isnan(zlo))
                    continue;
            }
#pragma unroll 1
            for (int kk = 0; kk < 3; ++kk) {
                const int k = kk - 1;
                const float kz = (float)k * P.boxf[2];
                int jlo, jhi;
                if (PREWIN) {  // clip the column-b window to this tile
                    const int lo = kk == 0 ? wl0 : (kk == 1 ? wl1 : wl2);
                    const int hi = kk == 0 ? wh0 : (kk == 1 ? wh1 : wh2);
                    jlo = max(lo, t0) - t0;
                    jhi = min(hi, t0 + nt) - t0;
                    if (jlo >= jhi)
                        continue;
                } else {
                    if (k < it.kmin || k > it.kmax)
                        continue;
                    const float wlo = zlo - kz - dzw, whi = zhi - kz + dzw;
                    if (whi < zt_lo || wlo > zt_hi)
                        continue;
                    const int lp = kk == 0 ? lo_prev[0] : (kk == 1 ? lo_prev[1] : lo_prev[2]);
                    const int hp = kk == 0 ? hi_prev[0] : (kk == 1 ? hi_prev[1] : hi_prev[2]);
                    jlo = warp_bound_from(zkey, lp, nt, wlo, false, lane);
                    jhi = warp_bound_from(zkey, max(hp, jlo), nt, whi, true, lane);
                    if (kk == 0) {
                        lo_prev[0] = jlo;
                        hi_prev[0] = jhi;
                    } else if (kk == 1) {
                        lo_prev[1] = jlo;
                        hi_prev[1] = jhi;
                    } else {
                        lo_prev[2] = jlo;
                        hi_prev[2] = jhi;
                    }
                }
                const bool tri = it.self && k == 0;
                if (tri)
                    jlo = max(jlo, ib + 1 - t0);
                if (jlo >= jhi)
                    continue;
                pending += (unsigned)((jhi - jlo) / (64 / I) + 4) * 2u * PP;
#pragma unroll
                for (int q = 0; q < PP; ++q) {
                    const float zh = __fsub_rn(zq[q], kz);
                    ZH[q] = pack2(zh, zh);
                    if (RL) {
                        const float lz = __fsub_rn(__fadd_rn(lzq, two_sum_err(zq[q], -kz, zh)),
                                                   (float)k * dLz);
                        LZ = pack2(lz, lz);
                    }
                }
                S.Sz = k == 0 ? 0.0 : (k > 0 ? P.g.box[2] : -P.g.box[2]);
                if (W)
                    A.wsj = P.B.ws + t0;
                if (tri) {
                    if (lin)
                        sweep32<I, PP, true, EVALS, VERIFY, true, W, RV, RL>(
                            smem, S, hl, jlo, jhi, jj, XH, YH, ZH, iv, vv, n_eval, n_rck, n_viol,
                            A, wi, st.wpend, LX, LY, LZ);
                    else
                        sweep32<I, PP, true, EVALS, VERIFY, false, W, RV, RL>(
                            smem, S, hl, jlo, jhi, jj, XH, YH, ZH, iv, vv, n_eval, n_rck, n_viol,
                            A, wi, st.wpend, LX, LY, LZ);
                } else {
                    if (lin)
                        sweep32<I, PP, false, EVALS, VERIFY, true, W, RV, RL>(
                            smem, S, hl, jlo, jhi, jj, XH, YH, ZH, iv, vv, n_eval, n_rck, n_viol,
                            A, wi, st.wpend, LX, LY, LZ);
                    else
                        sweep32<I, PP, false, EVALS, VERIFY, false, W, RV, RL>(
                            smem, S, hl, jlo, jhi, jj, XH, YH, ZH, iv, vv, n_eval, n_rck, n_viol,
                            A, wi, st.wpend, LX, LY, LZ);
                }
            }
            // keep every shared u32 count far from overflow (WARPS / HC warps add to a copy)
            if (!(W || RV) && pending > (1u << 30) / (WARPS / HC)) {
                __syncwarp();
                if (HC == WARPS)
                    warp_flush(hw, nb, P.hist, lane);
                else
                    warp_flush_shared(hw, nb, P.hist, lane);
                pending = 0;
            }
        }
    }

    static __device__ __forceinline__ void fini(const PairParams &P, unsigned char *smem, PathState &st)
    {
        // I * PP primaries per chunk (lane ii = lane % I holds primaries ii, ii + I,
        // ...); jj = lane / I picks the pair of secondaries.
        const int nb = P.nbins;
        uint32_t *hist = reinterpret_cast<uint32_t *>(smem + HIST_OFF);

        const int tid = threadIdx.x, lane = tid & 31;
        u64 &n_eval = st.n_eval;
        u64 &n_rck = st.n_rck;
        u64 &n_viol = st.n_viol;

        if (W || RV) {
            // the lane's last rows, then the CTA's 64-bit sums -> global
            const int plane = WARPS * (nb + 2) * 32, warp = tid >> 5;
            WAcc A;
            A.cnt = hist + (warp * (nb + 2) + 1) * 32 + lane;
            A.wq = A.cnt + plane;
            A.rq = A.cnt + (W ? 2 : 1) * plane;
            A.g = P.wscratch + ((long long)blockIdx.x * THREADS + tid) * 3 * nb;
            A.nb = nb;
            wacc_flush<W, RV>(A);
            __threadfence_block();
            __syncthreads();
            const float *sr = reinterpret_cast<const float *>(hist + (1 + (W ? 1 : 0) + (RV ? 1 : 0)) * plane) + 1;
            const float sw = W ? pow2_floor(2097152.0f / wmax_pair(P)) : 1.0f;
            const long long *gb = P.wscratch + (long long)blockIdx.x * THREADS * 3 * nb;
            for (int bn = tid; bn < nb; bn += THREADS) {
                long long c = 0, wsum = 0, rsum = 0;
                for (int t = 0; t < THREADS; ++t) {
                    c += gb[((long long)t * nb + bn) * 3];
                    wsum += gb[((long long)t * nb + bn) * 3 + 1];
                    rsum += gb[((long long)t * nb + bn) * 3 + 2];
                }
                if (c) {
                    atomicAdd(&P.hist[bn], (u64)c);
                    if (W)
                        atomicAdd(&P.wsum[bn], (double)wsum / (double)sw);
                    if (RV)
                        atomicAdd(&P.rsum[bn], (double)rsum / (double)sr[bn]);
                }
            }
        } else {
            __syncthreads();
            for (int bn = tid; bn < nb; bn += THREADS) {
                u64 sum = 0;
                for (int w = 0; w < HC; ++w)
                    for (int l = 0; l < 32; ++l)
                        sum += hist[(w * (nb + 2) + 1 + bn) * 32 + l];
                if (sum)
                    atomicAdd(&P.hist[bn], sum);
            }
        }
        n_eval = warp_sum_u64(n_eval);
        n_rck = warp_sum_u64(n_rck);
        n_viol = warp_sum_u64(n_viol);
        if (lane == 0) {
            if (n_eval)
                atomicAdd(&P.diag[1], n_eval);
            if (n_rck)
                atomicAdd(&P.diag[2], n_rck);
            if (n_viol)
                atomicAdd(&P.diag[3], n_viol);
        }
    }
};

__device__ __forceinline__ float sqrt_approx(float v)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// ============================================================ binary64 kernel
template <int I, bool EVALS, bool WACC>
struct Xi64Path {
    static __device__ __forceinline__ void init(const PairParams &P, unsigned char *smem)
    {
        const int nb = P.nbins;
        const Smem64 L = smem64_layout(P.tile_max, nb, 0, WARPS * (nb + 1) * 32);
        double *E2 = reinterpret_cast<double *>(smem + L.e2);
        uint32_t *hist = reinterpret_cast<uint32_t *>(smem + L.hist);
        double *acc = WACC ? reinterpret_cast<double *>(smem + P.acc_off) : nullptr;  // [warp][bin][2]

        const int tid = threadIdx.x;
        for (int q = tid; q <= nb; q += THREADS)
            E2[q] = P.E2[q];
        for (int q = tid; q < WARPS * (nb + 1) * 32; q += THREADS)
            hist[q] = 0u;
        if (WACC)
            for (int q = tid; q < WARPS * nb * 2; q += THREADS)
                acc[q] = 0.0;
    }

    static __device__ __forceinline__ bool item(const PairParams &P, const Item &it,
                                                unsigned char *smem, PathState &st)
    {
        constexpr int J = 32 / I;
        const int nb = P.nbins;
        const Smem64 L = smem64_layout(P.tile_max, nb, 0, WARPS * (nb + 1) * 32);
        uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
        double4_32a *tile = reinterpret_cast<double4_32a *>(smem + L.tile);
        double *E2 = reinterpret_cast<double *>(smem + L.e2);
        uint32_t *hist = reinterpret_cast<uint32_t *>(smem + L.hist);
        double *acc = WACC ? reinterpret_cast<double *>(smem + P.acc_off) : nullptr;  // [warp][bin][2]

        const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
        unsigned &phase = st.phase;
        u64 &n_eval = st.n_eval;
        unsigned &pending = st.pending;

        uint32_t *hw = hist + warp * (nb + 1) * 32;
        uint32_t *hl = hw + lane;
        const int ii = lane % I, jj = lane / I;
        const double qnan = __longlong_as_double(0x7ff8000000000000ll);

        const double dzw = __dadd_rn(it.dzmax, 1e-9 * (P.rz + P.g.box[2] + 1.0));
        const int nchunks = (it.a1 - it.a0 + I - 1) / I;

        for (int t0 = it.b0; t0 < it.b1; t0 += P.tile_max) {
            const int nt = min(P.tile_max, it.b1 - t0);
            if (!stage_tile(tile, P.B.pos64 + t0, nt, 32, bar, phase, P.err, P.wait_ns)) {
                return false;
            }
            const double zt_lo = tile[0].z, zt_hi = tile[nt - 1].z;
            auto zkey = [&](int p) { return tile[p].z; };
            auto next_chunk = [&]() {  // chunks in increasing order, claimed by the warps
                int v = 0;
                if (lane == 0)
                    v = atomicAdd(reinterpret_cast<int *>(smem + CLAIM_OFF), 1);
                return __shfl_sync(FULL, v, 0);
            };
            for (int c = next_chunk(); c < nchunks; c = next_chunk()) {
                const int ib = it.a0 + c * I;
                const int nvi = min(I, it.a1 - ib);
                const int i = ib + ii;
                const bool vi = ii < nvi;
                double4_32a pi = make_double4_32a(qnan, qnan, qnan, qnan);
                if (vi)
                    pi = P.A.pos64[i];  // column padding entries are NaN
                const double zlo = __shfl_sync(FULL, pi.z, 0);
                double zhi = pi.z;
    #pragma unroll
                for (int o = 1; o < I; o <<= 1) {  // largest real z of the chunk
                    const double t = __shfl_xor_sync(FULL, zhi, o);
                    zhi = (isnan(zhi) || t > zhi) ? t : zhi;
                }
                if (isnan(zlo))
                    continue;
                for (int k = it.kmin; k <= it.kmax; ++k) {
                    const double kz = k * P.g.box[2];
                    const double wlo = zlo - kz - dzw, whi = zhi - kz + dzw;
                    if (whi < zt_lo || wlo > zt_hi)
                        continue;
                    int jlo = warp_bound(zkey, nt, wlo, false, lane);
                    const int jhi = warp_bound(zkey, nt, whi, true, lane);
                    const bool tri = it.self && k == 0;
                    if (tri)
                        jlo = max(jlo, ib + 1 - t0);
                    if (jlo >= jhi)
                        continue;
                    pending += (unsigned)((jhi - jlo + J - 1) / J);
                    const bool noshift = it.Sx == 0.0 && it.Sy == 0.0 && kz == 0.0;
                    for (int jb = jlo; jb < jhi; jb += J) {
                        const int j = jb + jj;
                        const double4_32a pj = tile[j];
                        const bool live = !tri || (t0 + j > i);
                        if (EVALS)
                            n_eval += (vi && j < jhi && live) ? 1ull : 0ull;
                        double r2;
                        if (noshift)
                            r2 = plain_r2(pi, pj);
                        else
                            r2 = canon_r2(pi, pj, it.Sx, it.Sy, kz);
                        if (!live)
                            r2 = qnan;
                        const int kb = bin_f64(r2, E2, nb);
                        if (kb >= 0) {
                            hl[kb * 32] += 1u;
                            if (WACC) {  // Code 1's weight; the oracle's product and sqrt
                                double *aw = acc + (warp * nb + kb) * 2;
                                const double pw = P.weighted ? __dmul_rn(pi.w, pj.w) : 1.0;
                                atomicAdd(aw, pw);
                                if (P.want_r)
                                    atomicAdd(aw + 1, __dmul_rn(__dsqrt_rn(r2), pw));
                            }
                        }
                    }
                }
                if (pending > (1u << 30)) {
                    warp_flush(hw, nb, P.hist, lane);
                    pending = 0;
                }
            }
        }
        return true;
    }

    static __device__ __forceinline__ void fini(const PairParams &P, unsigned char *smem, PathState &st)
    {
        const int nb = P.nbins;
        const Smem64 L = smem64_layout(P.tile_max, nb, 0, WARPS * (nb + 1) * 32);
        uint32_t *hist = reinterpret_cast<uint32_t *>(smem + L.hist);
        double *acc = WACC ? reinterpret_cast<double *>(smem + P.acc_off) : nullptr;  // [warp][bin][2]

        const int tid = threadIdx.x, lane = tid & 31;
        u64 &n_eval = st.n_eval;

        __syncthreads();
        for (int bn = tid; bn < nb; bn += THREADS) {
            u64 sum = 0;
            double ws = 0.0, rs = 0.0;
            for (int w = 0; w < WARPS; ++w) {
                for (int l = 0; l < 32; ++l)
                    sum += hist[(w * (nb + 1) + bn) * 32 + l];
                if (WACC) {
                    ws += acc[(w * nb + bn) * 2];
                    rs += acc[(w * nb + bn) * 2 + 1];
                }
            }
            if (sum) {
                atomicAdd(&P.hist[bn], sum);
                if (WACC) {
                    atomicAdd(&P.wsum[bn], ws);
                    if (P.want_r)
                        atomicAdd(&P.rsum[bn], rs);
                }
            }
        }
        n_eval = warp_sum_u64(n_eval);
        if (lane == 0 && n_eval)
            atomicAdd(&P.diag[1], n_eval);
    }
};

// ============================================================ DD(rp, pi) kernels
// rp^2 = dx^2 + dy^2 is binned like r^2 (bits-indexed table of float32
// thresholds with 2-component error bands).  pi = |dz| is binned by
// arithmetic, since its edges are uniform: t = |dz| * npibins / pimax has the
// pi edges at the integers.  With t' = t - 1/2 (one fma), adding 1.5 * 2^23
// rounds t' to the nearest integer m, which the sum's low mantissa bits hold;
// m = floor(t) unless t is within rounding of an integer, and the exact
// remainder d = t' - m tells that case apart (|d| close to 1/2).
constexpr float PI_MAGIC = 12582912.0f;        // 1.5 * 2^23: spacing 1 in [2^23, 2^24)
constexpr uint32_t PI_MAGIC_BITS = 0x4b400000u;  // its bit pattern

__device__ __forceinline__ u64 fadd2(u64 a, u64 b)
{
    u64 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ u64 fabs2(u64 a) { return a & 0x7fffffff7fffffffull; }

__device__ __forceinline__ void red_shared(uint32_t addr, uint32_t v)
{
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}

// Canonical binary64 rp^2 of one pair inside an rp band: rp bin or -1.
__device__ __noinline__ int recheck_rp64(const double *E2, int nb, const double4_32a *pa,
                                         const double4_32a *pb, int i, int j, double Sx, double Sy)
{
    const double dx = canon_comp(pa[i].x, pb[j].x, Sx);
    const double dy = canon_comp(pa[i].y, pb[j].y, Sy);
    return bin_f64(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), E2, nb);
}

// Canonical binary64 pi = |dz| of one pair near a pi edge: pi bin or -1.
__device__ __noinline__ int recheck_pi64(const double *Pe, int npi, const double4_32a *pa,
                                         const double4_32a *pb, int i, int j, double Sz)
{
    return bin_f64(fabs(canon_comp(pa[i].z, pb[j].z, Sz)), Pe, npi);
}

// Debug: do the float32 decisions (rp from thresholds, pi from the rounding)
// agree with binary64?  No claim inside a band.  (1 = violation)
__device__ __noinline__ int verify_rppi(float rp2, uint32_t m32, bool pflag, const float *thr,
                                        int nthr, int nb, int npi, const double *E2,
                                        const double *Pe, const double4_32a *pa,
                                        const double4_32a *pb, int i, int j, double Sx, double Sy,
                                        double Sz)
{
    int c = 0;
    while (c < nthr && thr[c] <= rp2)
        ++c;
    if ((c & 1) || pflag)
        return 0;
    const int k32 = (c >= 2 && c <= 2 * nb) ? (c - 2) >> 1 : -1;
    const int mm = m32 < (uint32_t)npi ? (int)m32 : -1;
    const int k64 = recheck_rp64(E2, nb, pa, pb, i, j, Sx, Sy);
    const int m64 = recheck_pi64(Pe, npi, pa, pb, i, j, Sz);
    const bool c32 = k32 >= 0 && mm >= 0, c64 = k64 >= 0 && m64 >= 0;
    return c32 != c64 || (c32 && (k32 != k64 || mm != m64));
}

// Per-window constants of the rp-pi sweep.
struct SweepRP {
    int t0, nb, npi;
    uint32_t u0, lut_last;
    int shift, nthr;
    int lin;       // rp^2 table cells linear (scale lscale) or logarithmic
    float lscale;
    uint32_t hbase, rowb;  // shared address of this warp's histogram copy; bytes per rp row
    float pband;
    double *acc;           // weighted sums: this copy's binary64 [slot][w, r w] (or NULL)
    bool weighted, want_r;
    const float *xlj, *ylj;  // secondaries' coordinate residuals from tile element 0 (or NULL)
    const double4_32a *pa, *pb;
    double Sx, Sy, Sz;
};

// A pair whose rp table cell is flagged or whose t is near a pi edge: settle
// both decisions exactly, undo the main path's increment (at addr_main) and
// add the pair to its true slot.  Returns 1 if binary64 was needed.
// The primary's side of a pair for the residual correction of its rp: the
// primary's shifted float32 coordinates and its residuals after the shift.
struct PrimRL {
    float xh, yh, lx, ly;
};

// Binary64 accumulation of one counted pair's weight and rp * weight.  With the
// coordinates' float32 rounding residuals (gridding stores them for float64
// inputs or an open box) rp^2 is corrected to first order, as the float32 DD(r)
// path corrects r^2: rp^2 = rp2~ + 2 (dx~ (r_xj - r_xi') + dy~ (r_yj - r_yi')),
// dx~ the float32 difference of the main path recomputed from the staged tile.
__device__ __forceinline__ void acc_rppi(const unsigned char *smem, const SweepRP &S, int slot,
                                         float pw, float rp2, int jl, const PrimRL &R)
{
    atomicAdd(S.acc + 2 * slot, (double)pw);
    if (S.want_r) {
        if (S.xlj) {
            const float *tx = reinterpret_cast<const float *>(smem + TX_OFF);
            const float dx = __fsub_rn(tx[jl], R.xh), dy = __fsub_rn(tx[jl + TSTRIDE / 4], R.yh);
            rp2 = __fmaf_rn(2.0f, __fmaf_rn(dy, S.ylj[jl] - R.ly, dx * (S.xlj[jl] - R.lx)), rp2);
        }
        atomicAdd(S.acc + 2 * slot + 1, (double)(sqrt_approx(rp2) * pw));
    }
}

template <bool WACC>
__device__ __forceinline__ int resolve_rppi(const unsigned char *smem, const SweepRP &S, uint32_t e,
                                            float rp2, uint32_t m_main, bool pflag,
                                            uint32_t addr_main, int i, int jg, float pw,
                                            const PrimRL &R = PrimRL{0.0f, 0.0f, 0.0f, 0.0f})
{
    int k, re = 0;
    if (e > (uint32_t)S.nb) {
        const float *T = reinterpret_cast<const float *>(smem + THR_OFF);
        const int c = thr_count(T, S.nthr, rp2);
        if (c & 1) {
            k = recheck_rp64(reinterpret_cast<const double *>(smem + E2_OFF), S.nb, S.pa, S.pb, i,
                             jg, S.Sx, S.Sy);
            re = 1;
        } else {
            k = (c >= 2 && c <= 2 * S.nb) ? (c - 2) >> 1 : -1;
        }
    } else {
        k = e < (uint32_t)S.nb ? (int)e : -1;
    }
    if (k < 0)  // the main path used the dummy row
        return re;
    int m;
    if (pflag) {
        m = recheck_pi64(reinterpret_cast<const double *>(smem + RPPI_P_OFF), S.npi, S.pa, S.pb, i,
                         jg, S.Sz);
        re = 1;
    } else {
        m = m_main < (uint32_t)S.npi ? (int)m_main : -1;
    }
    red_shared(addr_main, 0xffffffffu);
    if (m >= 0) {
        red_shared(S.hbase + (uint32_t)k * S.rowb + (uint32_t)m * 4u, 1u);
        if (WACC)
            acc_rppi(smem, S, k * (S.npi + 1) + m, pw, rp2, jg - S.t0, R);
    }
    return re;
}

// Sweep one window of the staged tile (lane layout as in sweep32): per pair
// rp^2 and t' = |dz| * s - 1/2 in packed float32, the rp table byte, the pi
// index from the rounding, one shared atomic into the warp's 2-D histogram
// copy; one warp-uniform check for flagged pairs per iteration.
template <int I, bool TRI, bool EVALS, bool VERIFY, bool WACC, bool LIN>
__device__ __forceinline__ void sweep_rppi32(unsigned char *smem, const SweepRP &S, int jlo, int jhi,
                                             int jj, u64 XH, u64 YH, u64 ZH, u64 SC, u64 WH, int i,
                                             bool vi, u64 &n_eval, u64 &n_rck, u64 &n_viol,
                                             const PrimRL &R)
{
    const float qnan = __int_as_float(0x7fc00000);
    const u64 MH = pack2(-0.5f, -0.5f), MG = pack2(PI_MAGIC, PI_MAGIC);
    const uint32_t npiu = (uint32_t)S.npi, nbu = (uint32_t)S.nb;
    const int jstart = jlo & ~1;
    constexpr int JS = 64 / I;
    const int nit = (jhi - jstart + 2 * JS - 1) / (2 * JS);
    const unsigned char *p = smem + TX_OFF + (jstart + 2 * jj) * 4;
    int jA = jstart + 2 * jj;
    for (int it = 0; it < nit; ++it, p += 8 * JS, jA += 2 * JS) {
        const u64 xA = *reinterpret_cast<const u64 *>(p);
        const u64 yA = *reinterpret_cast<const u64 *>(p + TSTRIDE);
        const u64 zA = *reinterpret_cast<const u64 *>(p + 2 * TSTRIDE);
        const u64 xB = *reinterpret_cast<const u64 *>(p + 4 * JS);
        const u64 yB = *reinterpret_cast<const u64 *>(p + 4 * JS + TSTRIDE);
        const u64 zB = *reinterpret_cast<const u64 *>(p + 4 * JS + 2 * TSTRIDE);
        u64 dx = fsub2(xA, XH), dy = fsub2(yA, YH);
        const u64 rA = ffma2(dy, dy, fmul2(dx, dx));
        const u64 tA = ffma2(fabs2(fsub2(zA, ZH)), SC, MH);
        dx = fsub2(xB, XH);
        dy = fsub2(yB, YH);
        const u64 rB = ffma2(dy, dy, fmul2(dx, dx));
        const u64 tB = ffma2(fabs2(fsub2(zB, ZH)), SC, MH);
        const u64 qA = fadd2(tA, MG), qB = fadd2(tB, MG);
        const u64 fA = fsub2(tA, fsub2(qA, MG)), fB = fsub2(tB, fsub2(qB, MG));
        float a0, a1, b0, b1, fa0, fa1, fb0, fb1, qa0, qa1, qb0, qb1;
        unpack2(rA, a0, a1);
        unpack2(rB, b0, b1);
        unpack2(fA, fa0, fa1);
        unpack2(fB, fb0, fb1);
        unpack2(qA, qa0, qa1);
        unpack2(qB, qb0, qb1);
        const int gA = S.t0 + jA, gB = gA + JS;
        bool la0 = true, la1 = true, lb0 = true, lb1 = true;
        if (TRI) {
            la0 = gA > i;
            la1 = gA + 1 > i;
            lb0 = gB > i;
            lb1 = gB + 1 > i;
            a0 = la0 ? a0 : qnan;
            a1 = la1 ? a1 : qnan;
            b0 = lb0 ? b0 : qnan;
            b1 = lb1 ? b1 : qnan;
        }
        if (EVALS) {
            const int jB = jA + JS;
            n_eval += (u64)((vi && jA >= jlo && jA < jhi && la0) +
                            (vi && jA + 1 >= jlo && jA + 1 < jhi && la1) +
                            (vi && jB >= jlo && jB < jhi && lb0) +
                            (vi && jB + 1 >= jlo && jB + 1 < jhi && lb1));
        }
        const uint32_t ea0 = lut_entry<LIN>(smem, S.u0, S.shift, S.lut_last, S.lscale, a0);
        const uint32_t ea1 = lut_entry<LIN>(smem, S.u0, S.shift, S.lut_last, S.lscale, a1);
        const uint32_t eb0 = lut_entry<LIN>(smem, S.u0, S.shift, S.lut_last, S.lscale, b0);
        const uint32_t eb1 = lut_entry<LIN>(smem, S.u0, S.shift, S.lut_last, S.lscale, b1);
        const uint32_t ma0 = min(__float_as_uint(qa0) - PI_MAGIC_BITS, npiu);
        const uint32_t ma1 = min(__float_as_uint(qa1) - PI_MAGIC_BITS, npiu);
        const uint32_t mb0 = min(__float_as_uint(qb0) - PI_MAGIC_BITS, npiu);
        const uint32_t mb1 = min(__float_as_uint(qb1) - PI_MAGIC_BITS, npiu);
        const uint32_t ha0 = S.hbase + min(ea0, nbu) * S.rowb + ma0 * 4u;
        const uint32_t ha1 = S.hbase + min(ea1, nbu) * S.rowb + ma1 * 4u;
        const uint32_t hb0 = S.hbase + min(eb0, nbu) * S.rowb + mb0 * 4u;
        const uint32_t hb1 = S.hbase + min(eb1, nbu) * S.rowb + mb1 * 4u;
        red_shared(ha0, 1u);
        red_shared(ha1, 1u);
        red_shared(hb0, 1u);
        red_shared(hb1, 1u);
        const bool pa0 = fabsf(fa0) > S.pband, pa1 = fabsf(fa1) > S.pband;
        const bool pb0 = fabsf(fb0) > S.pband, pb1 = fabsf(fb1) > S.pband;
        float wa0 = 1.0f, wa1 = 1.0f, wb0 = 1.0f, wb1 = 1.0f;
        if (WACC) {
            if (S.weighted) {
                const unsigned char *pw8 = smem + XIW_W_OFF + (p - (smem + TX_OFF));
                unpack2(fmul2(*reinterpret_cast<const u64 *>(pw8), WH), wa0, wa1);
                unpack2(fmul2(*reinterpret_cast<const u64 *>(pw8 + 4 * JS), WH), wb0, wb1);
            }
            // pairs settled by the float32 path; flagged ones are added when resolved
            if (!pa0 && ea0 < nbu && ma0 < npiu)
                acc_rppi(smem, S, (int)(ea0 * (npiu + 1) + ma0), wa0, a0, jA, R);
            if (!pa1 && ea1 < nbu && ma1 < npiu)
                acc_rppi(smem, S, (int)(ea1 * (npiu + 1) + ma1), wa1, a1, jA + 1, R);
            if (!pb0 && eb0 < nbu && mb0 < npiu)
                acc_rppi(smem, S, (int)(eb0 * (npiu + 1) + mb0), wb0, b0, jA + JS, R);
            if (!pb1 && eb1 < nbu && mb1 < npiu)
                acc_rppi(smem, S, (int)(eb1 * (npiu + 1) + mb1), wb1, b1, jA + JS + 1, R);
        }
        const bool ga0 = ea0 > nbu || pa0, ga1 = ea1 > nbu || pa1;
        const bool gb0 = eb0 > nbu || pb0, gb1 = eb1 > nbu || pb1;
        if (__any_sync(FULL, ga0 || ga1 || gb0 || gb1)) {
            if (ga0)
                n_rck += resolve_rppi<WACC>(smem, S, ea0, a0, ma0, pa0, ha0, i, gA, wa0, R);
            if (ga1)
                n_rck += resolve_rppi<WACC>(smem, S, ea1, a1, ma1, pa1, ha1, i, gA + 1, wa1, R);
            if (gb0)
                n_rck += resolve_rppi<WACC>(smem, S, eb0, b0, mb0, pb0, hb0, i, gB, wb0, R);
            if (gb1)
                n_rck += resolve_rppi<WACC>(smem, S, eb1, b1, mb1, pb1, hb1, i, gB + 1, wb1, R);
        }
        if (VERIFY) {
            const float *T = reinterpret_cast<const float *>(smem + THR_OFF);
            const double *E2 = reinterpret_cast<const double *>(smem + E2_OFF);
            const double *Pe = reinterpret_cast<const double *>(smem + RPPI_P_OFF);
            const float dv[4] = {a0, a1, b0, b1};
            const uint32_t mv[4] = {ma0, ma1, mb0, mb1};
            const bool pv[4] = {pa0, pa1, pb0, pb1};
            const int gv[4] = {gA, gA + 1, gB, gB + 1};
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (vi && !isnan(dv[q]))
                    n_viol += verify_rppi(dv[q], mv[q], pv[q], T, S.nthr, S.nb, S.npi, E2, Pe, S.pa,
                                          S.pb, i, gv[q], S.Sx, S.Sy, S.Sz);
        }
    }
}

// Move one histogram copy to the global histogram.  Counts are read as
// signed 32-bit values: a warp may undo an increment (resolve_rppi) after
// another warp sharing the copy has flushed it.
__device__ void flush_rppi(uint32_t *hc, int nb, int npi, unsigned long long *ghist, int lane)
{
    const int row = npi + 1;
    for (int s = lane; s < nb * row; s += 32) {
        const int k = s / row, m = s - k * row;
        if (m == npi)
            continue;
        const int v = (int)atomicExch(&hc[s], 0u);
        if (v)
            atomicAdd(&ghist[k * npi + m], (u64)(long long)v);
    }
}

// All copies of the CTA's histograms (and binary64 sums, if acc) -> global
// (after the last __syncthreads).
__device__ void merge_rppi(const PairParams &P, const uint32_t *hist, const double *acc, int rows,
                           int row0 = 0)
{
    const int nb = P.nbins, npi = P.npibins, row = npi + 1, copy = rows * row;
    for (int s = threadIdx.x; s < nb * npi; s += THREADS) {
        const int k = s / npi, m = s - k * npi;
        long long sum = 0;
        double ws = 0.0, rs = 0.0;
        for (int c = 0; c < P.hcopies; ++c) {
            const int q = c * copy + k * row + m;  // binary64 sums have no row -1
            sum += (int)hist[q + row0 * row];
            if (acc) {
                ws += acc[2 * q];
                rs += acc[2 * q + 1];
            }
        }
        if (sum) {
            atomicAdd(&P.hist[s], (u64)sum);
            if (acc) {
                atomicAdd(&P.wsum[s], ws);
                if (P.want_r)
                    atomicAdd(&P.rsum[s], rs);
            }
        }
    }
}

template <int I, bool EVALS, bool VERIFY, bool WACC>
struct Rppi32Path {
    static __device__ __forceinline__ void init(const PairParams &P, unsigned char *smem)
    {
        const int nb = P.nbins, npi = P.npibins;
        float *thr = reinterpret_cast<float *>(smem + THR_OFF);
        double *E2 = reinterpret_cast<double *>(smem + E2_OFF);
        double *Pe = reinterpret_cast<double *>(smem + RPPI_P_OFF);
        uint32_t *hist = reinterpret_cast<uint32_t *>(smem + P.hist_off);
        double *acc = WACC ? reinterpret_cast<double *>(smem + P.acc_off) : nullptr;
        const int copy = rppi32_rows(nb) * (npi + 1);

        const int tid = threadIdx.x;
        for (int q = tid; q < P.lut_n; q += THREADS)
            smem[LUT_OFF + q] = P.lut[q];
        for (int q = tid; q < P.nthr; q += THREADS)
            thr[q] = P.thr[q];
        for (int q = tid; q <= nb; q += THREADS)
            E2[q] = P.E2[q];
        for (int q = tid; q <= npi; q += THREADS)
            Pe[q] = P.P[q];
        for (int q = tid; q < P.hcopies * copy; q += THREADS)
            hist[q] = 0u;
        if (WACC)
            for (int q = tid; q < 2 * P.hcopies * copy; q += THREADS)
                acc[q] = 0.0;
    }

    static __device__ __forceinline__ bool item(const PairParams &P, const Item &it,
                                                unsigned char *smem, PathState &st)
    {
        const int nb = P.nbins, npi = P.npibins;
        uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
        const float *tz = reinterpret_cast<const float *>(smem + TX_OFF + 2 * TSTRIDE);
        uint32_t *hist = reinterpret_cast<uint32_t *>(smem + P.hist_off);
        double *acc = WACC ? reinterpret_cast<double *>(smem + P.acc_off) : nullptr;
        const int copy = rppi32_rows(nb) * (npi + 1);

        const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
        unsigned &phase = st.phase;
        u64 &n_eval = st.n_eval;
        u64 &n_rck = st.n_rck;
        u64 &n_viol = st.n_viol;
        unsigned &pending = st.pending;

        uint32_t *hc = hist + (warp % P.hcopies) * copy + (npi + 1);  // row 0 of the warp's copy
        const int ii = lane % I, jj = lane / I;
        SweepRP S;
        S.nb = nb;
        S.npi = npi;
        S.u0 = P.u0;
        S.lut_last = (uint32_t)(P.lut_n - 1);
        S.shift = P.lut_shift;
        S.nthr = P.nthr;
        S.lin = P.lut_lin;
        S.lscale = P.lut_scale;
        S.hbase = smem_u32(hc);
        S.rowb = (uint32_t)(npi + 1) * 4u;
        S.pband = P.pband;
        S.pa = P.A.pos64;
        S.pb = P.B.pos64;
        S.acc = WACC ? acc + 2 * (warp % P.hcopies) * copy : nullptr;
        S.weighted = WACC && P.weighted;
        S.want_r = WACC && P.want_r;
        // rp of the mean separations from residual-corrected rp^2 when the gridding
        // stored the coordinates' float32 rounding residuals
        const bool rl = S.want_r && P.B.xl != nullptr;
        const u64 SC = pack2(P.pscale, P.pscale);
        const unsigned flush_at = (1u << 30) / (unsigned)(WARPS / P.hcopies);
        const float qnan = __int_as_float(0x7fc00000);

        const float dzw = __fadd_ru(__double2float_ru(it.dzmax), P.zslack);
        const float Sxf = __double2float_rn(it.Sx), Syf = __double2float_rn(it.Sy);
        // the roundings of the periodic shifts, S - fl32(S)
        const float dSx = rl ? __double2float_rn(__dsub_rn(it.Sx, (double)Sxf)) : 0.0f;
        const float dSy = rl ? __double2float_rn(__dsub_rn(it.Sy, (double)Syf)) : 0.0f;
        S.Sx = it.Sx;
        S.Sy = it.Sy;
        const int nchunks = (it.a1 - it.a0 + I - 1) / I;

        for (int t0 = it.b0; t0 < it.b1; t0 += TILE32) {
            const int nt = min(TILE32, it.b1 - t0);
            if (!stage_tiles32(smem, P.B, t0, nt, bar, phase, P.err, P.wait_ns, S.weighted)) {
                return false;
            }
            S.t0 = t0;
            S.xlj = rl ? P.B.xl + t0 : nullptr;
            S.ylj = rl ? P.B.yl + t0 : nullptr;
            const float zt_lo = tz[0];
            float zt_hi = tz[nt - 1];
            if (isnan(zt_hi))
                zt_hi = INFINITY;
            auto zkey = [&](int q) { return tz[q]; };
            int lo_prev[3] = {0, 0, 0}, hi_prev[3] = {0, 0, 0};

            auto next_chunk = [&]() {  // chunks in increasing order, claimed by the warps
                int v = 0;
                if (lane == 0)
                    v = atomicAdd(reinterpret_cast<int *>(smem + CLAIM_OFF), 1);
                return __shfl_sync(FULL, v, 0);
            };
            for (int c = next_chunk(); c < nchunks; c = next_chunk()) {
                const int ib = it.a0 + c * I;
                const int nvi = min(I, it.a1 - ib);
                const int i = ib + ii;
                float xi = qnan, yi = qnan, zi = qnan, wi = 1.0f, rx = 0.0f, ry = 0.0f;
                if (ii < nvi) {
                    xi = P.A.xs[i];
                    yi = P.A.ys[i];
                    zi = P.A.zs[i];
                    if (S.weighted)
                        wi = P.A.ws[i];
                    if (rl) {
                        rx = P.A.xl[i];
                        ry = P.A.yl[i];
                    }
                }
                const bool vi = !isnan(xi);
                const float xh = __fsub_rn(xi, Sxf), yh = __fsub_rn(yi, Syf);
                const u64 XH = pack2(xh, xh), YH = pack2(yh, yh), WH = pack2(wi, wi);
                // the primary's residuals after the shift: r_i + (x~ - S~ - x^) - (S - S~)
                PrimRL R{xh, yh, 0.0f, 0.0f};
                if (rl) {
                    R.lx = __fsub_rn(__fadd_rn(rx, two_sum_err(xi, -Sxf, xh)), dSx);
                    R.ly = __fsub_rn(__fadd_rn(ry, two_sum_err(yi, -Syf, yh)), dSy);
                }
                const float zlo = __shfl_sync(FULL, zi, 0);
                float zhi = zi;
    #pragma unroll
                for (int o = 1; o < I; o <<= 1) {
                    const float t = __shfl_xor_sync(FULL, zhi, o);
                    zhi = (isnan(zhi) || t > zhi) ? t : zhi;
                }
                if (isnan(zlo))
                    continue;

    #pragma unroll
                for (int kk = 0; kk < 3; ++kk) {
                    const int k = kk - 1;
                    if (k < it.kmin || k > it.kmax)
                        continue;
                    const float kz = (float)k * P.boxf[2];
                    const float wlo = zlo - kz - dzw, whi = zhi - kz + dzw;
                    if (whi < zt_lo || wlo > zt_hi)
                        continue;
                    int jlo = warp_bound_from(zkey, lo_prev[kk], nt, wlo, false, lane);
                    const int jhi = warp_bound_from(zkey, max(hi_prev[kk], jlo), nt, whi, true, lane);
                    lo_prev[kk] = jlo;
                    hi_prev[kk] = jhi;
                    const bool tri = it.self && k == 0;
                    if (tri)
                        jlo = max(jlo, ib + 1 - t0);
                    if (jlo >= jhi)
                        continue;
                    pending += (unsigned)((jhi - jlo) / (64 / I) + 4) * 64u;
                    const float zh = __fsub_rn(zi, kz);
                    const u64 ZH = pack2(zh, zh);
                    S.Sz = k == 0 ? 0.0 : (k > 0 ? P.g.box[2] : -P.g.box[2]);
                    if (tri) {
                        if (S.lin)
                            sweep_rppi32<I, true, EVALS, VERIFY, WACC, true>(
                                smem, S, jlo, jhi, jj, XH, YH, ZH, SC, WH, i, vi, n_eval, n_rck, n_viol, R);
                        else
                            sweep_rppi32<I, true, EVALS, VERIFY, WACC, false>(
                                smem, S, jlo, jhi, jj, XH, YH, ZH, SC, WH, i, vi, n_eval, n_rck, n_viol, R);
                    } else {
                        if (S.lin)
                            sweep_rppi32<I, false, EVALS, VERIFY, WACC, true>(
                                smem, S, jlo, jhi, jj, XH, YH, ZH, SC, WH, i, vi, n_eval, n_rck, n_viol, R);
                        else
                            sweep_rppi32<I, false, EVALS, VERIFY, WACC, false>(
                                smem, S, jlo, jhi, jj, XH, YH, ZH, SC, WH, i, vi, n_eval, n_rck, n_viol, R);
                    }
                }
                if (pending > flush_at) {  // keep every shared u32 count far from overflow
                    __syncwarp();
                    flush_rppi(hc, nb, npi, P.hist, lane);
                    pending = 0;
                }
            }
        }
        return true;
    }

    static __device__ __forceinline__ void fini(const PairParams &P, unsigned char *smem, PathState &st)
    {

        uint32_t *hist = reinterpret_cast<uint32_t *>(smem + P.hist_off);
        double *acc = WACC ? reinterpret_cast<double *>(smem + P.acc_off) : nullptr;

        const int tid = threadIdx.x, lane = tid & 31;
        u64 &n_eval = st.n_eval;
        u64 &n_rck = st.n_rck;
        u64 &n_viol = st.n_viol;

        __syncthreads();
        merge_rppi(P, hist, acc, rppi32_rows(P.nbins), 1);
        n_eval = warp_sum_u64(n_eval);
        n_rck = warp_sum_u64(n_rck);
        n_viol = warp_sum_u64(n_viol);
        if (lane == 0) {
            if (n_eval)
                atomicAdd(&P.diag[1], n_eval);
            if (n_rck)
                atomicAdd(&P.diag[2], n_rck);
            if (n_viol)
                atomicAdd(&P.diag[3], n_viol);
        }
    }
};

// A pair recorded by sweep_rppi32_pp: recompute rp^2 and t' from the staged
// tile with the same IEEE operations as the packed main path, then settle it
// as resolve_rppi does (the main path added it at addr_main).
template <bool LIN>
__device__ __forceinline__ int resolve_local_rppi(const unsigned char *smem, const SweepRP &S,
                                                  float xh, float yh, float zh, float s,
                                                  int i, int jl)
{
    const float *tx = reinterpret_cast<const float *>(smem + TX_OFF);
    const float dx = __fsub_rn(tx[jl], xh);
    const float dy = __fsub_rn(tx[jl + TSTRIDE / 4], yh);
    const float dz = __fsub_rn(tx[jl + TSTRIDE / 2], zh);
    const float rp2 = __fmaf_rn(dy, dy, __fmul_rn(dx, dx));
    const float t = __fmaf_rn(fabsf(dz), s, -0.5f);
    const float q = __fadd_rn(t, PI_MAGIC);
    const float f = __fsub_rn(t, __fsub_rn(q, PI_MAGIC));
    // the entry as the main path loaded it (sign-extended: flagged = -1)
    const uint32_t e = (uint32_t)(int)(signed char)lut_entry<LIN>(smem, S.u0, S.shift, S.lut_last,
                                                                  S.lscale, rp2);
    const uint32_t m = min(__float_as_uint(q) - PI_MAGIC_BITS, (uint32_t)S.npi);
    const uint32_t addr = S.hbase + e * S.rowb + m * 4u;  // as the main path added it
    return resolve_rppi<false>(smem, S, e, rp2, m, fabsf(f) > S.pband, addr, i, S.t0 + jl, 1.0f);
}

// Sweep one window with PP primaries per lane (lane layout as in sweep32): per
// pair rp^2 and t' = |dz| s - 1/2 in packed float32, the rp table byte, the pi
// index from the rounding, one shared atomic into the warp's 2-D histogram copy.
// A pair whose rp cell is flagged, or whose t' lies within the error bound of
// a pi edge (|t' - round(t')| >= pband), sets a bit of the lane's mask; once
// per block of 8 steps a warp-uniform test settles the recorded pairs.
template <int I, int PP, bool TRI, bool EVALS, bool LIN>
__device__ __forceinline__ void sweep_rppi32_pp(unsigned char *smem, const SweepRP &S, int jlo,
                                                int jhi, int jj, const u64 *XH, const u64 *YH,
                                                const u64 *ZH, u64 SC, float sc, const int *iv,
                                                const bool *vv, u64 &n_eval, u64 &n_rck)
{
    const float qnan = __int_as_float(0x7fc00000);
    const u64 MH = pack2(-0.5f, -0.5f), MG = pack2(PI_MAGIC, PI_MAGIC);
    const u64 PB = pack2(S.pband, S.pband);
    const u64 LS = pack2(S.lscale, S.lscale), LM = pack2(LIN_MAGIC, LIN_MAGIC);
    const uint32_t npiu = (uint32_t)S.npi;
    // shared addresses of the rp table, the base folded into the clamp (as in sweep32)
    const uint32_t lutb = smem_u32(smem + LUT_OFF), lut_lo = lutb - LIN_MAGIC_BITS,
                   lut_hi = lutb + S.lut_last;
    const int jstart = jlo & ~1;
    constexpr int JS = 64 / I;
    const int nit = (jhi - jstart + 2 * JS - 1) / (2 * JS);
    for (int b0 = 0; b0 < nit; b0 += 8) {
        const int jAb = jstart + 2 * jj + b0 * 2 * JS;
        const uint32_t pb = smem_u32(smem + TX_OFF) + jAb * 4;
        const int tend = min(8, nit - b0);
        uint32_t fm[PP];
#pragma unroll
        for (int q = 0; q < PP; ++q)
            fm[q] = 0u;
        for (int t = 0; t < tend; ++t) {
            const uint32_t p = pb + t * 8 * JS;
            const u64 xA = lds64<0>(p);
            const u64 yA = lds64<TSTRIDE>(p);
            const u64 zA = lds64<2 * TSTRIDE>(p);
            const u64 xB = lds64<4 * JS>(p);
            const u64 yB = lds64<4 * JS + TSTRIDE>(p);
            const u64 zB = lds64<4 * JS + 2 * TSTRIDE>(p);
            const int jA = jAb + t * 2 * JS;
            const int gA = S.t0 + jA, gB = gA + JS;  // global indices of (a0, b0); a1, b1 are +1
            const int gv[4] = {gA, gA + 1, gB, gB + 1};
#pragma unroll
            for (int q = 0; q < PP; ++q) {
                u64 dx = fsub2(xA, XH[q]), dy = fsub2(yA, YH[q]);
                const u64 rA = ffma2(dy, dy, fmul2(dx, dx));
                const u64 tA = ffma2(fabs2(fsub2(zA, ZH[q])), SC, MH);
                dx = fsub2(xB, XH[q]);
                dy = fsub2(yB, YH[q]);
                const u64 rB = ffma2(dy, dy, fmul2(dx, dx));
                const u64 tB = ffma2(fabs2(fsub2(zB, ZH[q])), SC, MH);
                const u64 qA = fadd2(tA, MG), qB = fadd2(tB, MG);
                // pband - |t' - round(t')|: sign bit set = near a pi edge (a NaN
                // sentinel gives a positive NaN: never flagged)
                const u64 gA2 = fsub2(PB, fabs2(fsub2(tA, fsub2(qA, MG))));
                const u64 gB2 = fsub2(PB, fabs2(fsub2(tB, fsub2(qB, MG))));
                float r[4], qv[4], g[4];
                unpack2(rA, r[0], r[1]);
                unpack2(rB, r[2], r[3]);
                unpack2(qA, qv[0], qv[1]);
                unpack2(qB, qv[2], qv[3]);
                unpack2(gA2, g[0], g[1]);
                unpack2(gB2, g[2], g[3]);
                uint32_t cq[4];
                if (LIN) {
                    float c[4];
                    unpack2(ffma2(rA, LS, LM), c[0], c[1]);
                    unpack2(ffma2(rB, LS, LM), c[2], c[3]);
#pragma unroll
                    for (int k = 0; k < 4; ++k)  // the table byte's shared address
                        cq[k] = min(__float_as_uint(c[k]) + lut_lo, lut_hi);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        cq[k] = lutb + min((__float_as_uint(r[k]) >> S.shift) - S.u0, S.lut_last);
                }
                if (TRI) {  // pairs with j <= i: the out-of-range entry, never flagged
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        cq[k] = gv[k] > iv[q] ? cq[k] : lut_hi;
                        g[k] = gv[k] > iv[q] ? g[k] : 1.0f;
                    }
                }
                if (EVALS) {
                    const int jv[4] = {jA, jA + 1, jA + JS, jA + JS + 1};
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        n_eval += (vv[q] && jv[k] >= jlo && jv[k] < jhi && (!TRI || gv[k] > iv[q]))
                                      ? 1ull : 0ull;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t e = lds_entry(cq[k]);  // flagged: -1, the row before bin 0
                    const uint32_t m = min(__float_as_uint(qv[k]) - PI_MAGIC_BITS, npiu);
                    red_shared(S.hbase + e * S.rowb + m * 4u, 1u);
                    // pair (t, k) ends at bit 4 tend - 1 - (4 t + k): flagged rp cell or
                    // near a pi edge (sign of g)
                    fm[q] = push_sign(fm[q], e | __float_as_uint(g[k]));
                }
            }
        }
        uint32_t anyf = 0u;
#pragma unroll
        for (int q = 0; q < PP; ++q)
            anyf |= fm[q];
        if (__any_sync(FULL, anyf != 0u)) {
#pragma unroll
            for (int q = 0; q < PP; ++q) {
                float xh, yh, zh, tmp;
                unpack2(XH[q], xh, tmp);
                unpack2(YH[q], yh, tmp);
                unpack2(ZH[q], zh, tmp);
                uint32_t m = fm[q];
                while (m) {
                    const int bit = __ffs(m) - 1;
                    m &= m - 1u;
                    const int tk = 4 * tend - 1 - bit, t = tk >> 2, k = tk & 3;
                    const int jl = jAb + t * 2 * JS + ((k & 2) ? JS : 0) + (k & 1);
                    n_rck += resolve_local_rppi<LIN>(smem, S, xh, yh, zh, sc, iv[q], jl);
                }
            }
        }
    }
}

// Float32 DD(rp, pi) without sums: I x PP primaries per chunk (lane ii holds
// primaries ii, ii + I, ...), deferred flag resolution.  Tables, histograms and
// the merge are those of Rppi32Path.
template <int I, int PP, bool EVALS>
struct Rppi32PathPP {
    using Base = Rppi32Path<I, EVALS, false, false>;
    static __device__ __forceinline__ void init(const PairParams &P, unsigned char *smem)
    {
        Base::init(P, smem);
    }
    static __device__ __forceinline__ void fini(const PairParams &P, unsigned char *smem, PathState &st)
    {
        Base::fini(P, smem, st);
    }

    static __device__ __forceinline__ bool item(const PairParams &P, const Item &it,
                                                unsigned char *smem, PathState &st)
    {
        constexpr int CH = I * PP;
        const int nb = P.nbins, npi = P.npibins;
        uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
        const float *tz = reinterpret_cast<const float *>(smem + TX_OFF + 2 * TSTRIDE);
        uint32_t *hist = reinterpret_cast<uint32_t *>(smem + P.hist_off);
        const int copy = rppi32_rows(nb) * (npi + 1);

        const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
        unsigned &pending = st.pending;

        uint32_t *hc = hist + (warp % P.hcopies) * copy + (npi + 1);  // row 0 of the warp's copy
        const int ii = lane % I, jj = lane / I;
        SweepRP S;
        S.nb = nb;
        S.npi = npi;
        S.u0 = P.u0;
        S.lut_last = (uint32_t)(P.lut_n - 1);
        S.shift = P.lut_shift;
        S.nthr = P.nthr;
        S.lin = P.lut_lin;
        S.lscale = P.lut_scale;
        S.hbase = smem_u32(hc);
        S.rowb = (uint32_t)(npi + 1) * 4u;
        S.pband = P.pband;
        S.pa = P.A.pos64;
        S.pb = P.B.pos64;
        S.acc = nullptr;
        S.weighted = false;
        S.want_r = false;
        S.xlj = S.ylj = nullptr;
        const u64 SC = pack2(P.pscale, P.pscale);
        const unsigned flush_at = (1u << 30) / (unsigned)(WARPS / P.hcopies);
        const float qnan = __int_as_float(0x7fc00000);

        const float dzw = __fadd_ru(__double2float_ru(it.dzmax), P.zslack);
        const float Sxf = __double2float_rn(it.Sx), Syf = __double2float_rn(it.Sy);
        S.Sx = it.Sx;
        S.Sy = it.Sy;
        const int nchunks = (it.a1 - it.a0 + CH - 1) / CH;

        for (int t0 = it.b0; t0 < it.b1; t0 += TILE32) {
            const int nt = min(TILE32, it.b1 - t0);
            if (!stage_tiles32(smem, P.B, t0, nt, bar, st.phase, P.err, P.wait_ns))
                return false;
            S.t0 = t0;
            const float zt_lo = tz[0];
            float zt_hi = tz[nt - 1];
            if (isnan(zt_hi))
                zt_hi = INFINITY;
            auto zkey = [&](int q) { return tz[q]; };
            int lo_prev[3] = {0, 0, 0}, hi_prev[3] = {0, 0, 0};
            auto next_chunk = [&]() {  // chunks in increasing order, claimed by the warps
                int v = 0;
                if (lane == 0)
                    v = atomicAdd(reinterpret_cast<int *>(smem + CLAIM_OFF), 1);
                return __shfl_sync(FULL, v, 0);
            };
            for (int c = next_chunk(); c < nchunks; c = next_chunk()) {
                const int ib = it.a0 + c * CH;
                u64 XH[PP], YH[PP], ZH[PP];
                int iv[PP];
                bool vv[PP];
                float zq[PP];
                float zmax = qnan;
#pragma unroll
                for (int q = 0; q < PP; ++q) {
                    const int i = ib + q * I + ii;
                    float xi = qnan, yi = qnan, zi = qnan;
                    if (i < it.a1) {
                        xi = P.A.xs[i];
                        yi = P.A.ys[i];
                        zi = P.A.zs[i];
                    }
                    iv[q] = i;
                    vv[q] = !isnan(xi);  // chunk tail and column padding are NaN
                    const float xh = __fsub_rn(xi, Sxf), yh = __fsub_rn(yi, Syf);
                    XH[q] = pack2(xh, xh);
                    YH[q] = pack2(yh, yh);
                    zq[q] = zi;
                    zmax = (isnan(zmax) || zi > zmax) ? zi : zmax;
                }
                const float zlo = __shfl_sync(FULL, zq[0], 0);
                float zhi = zmax;
#pragma unroll
                for (int o = 1; o < I; o <<= 1) {  // largest real z of the chunk
                    const float t = __shfl_xor_sync(FULL, zhi, o);
                    zhi = (isnan(zhi) || t > zhi) ? t : zhi;
                }
                if (isnan(zlo))
                    continue;
#pragma unroll
                for (int kk = 0; kk < 3; ++kk) {
                    const int k = kk - 1;
                    if (k < it.kmin || k > it.kmax)
                        continue;
                    const float kz = (float)k * P.boxf[2];
                    const float wlo = zlo - kz - dzw, whi = zhi - kz + dzw;
                    if (whi < zt_lo || wlo > zt_hi)
                        continue;
                    int jlo = warp_bound_from(zkey, lo_prev[kk], nt, wlo, false, lane);
                    const int jhi = warp_bound_from(zkey, max(hi_prev[kk], jlo), nt, whi, true, lane);
                    lo_prev[kk] = jlo;
                    hi_prev[kk] = jhi;
                    const bool tri = it.self && k == 0;
                    if (tri)
                        jlo = max(jlo, ib + 1 - t0);
                    if (jlo >= jhi)
                        continue;
                    pending += (unsigned)((jhi - jlo) / (64 / I) + 4) * 2u * PP;
#pragma unroll
                    for (int q = 0; q < PP; ++q) {
                        const float zh = __fsub_rn(zq[q], kz);
                        ZH[q] = pack2(zh, zh);
                    }
                    S.Sz = k == 0 ? 0.0 : (k > 0 ? P.g.box[2] : -P.g.box[2]);
                    if (tri) {
                        if (S.lin)
                            sweep_rppi32_pp<I, PP, true, EVALS, true>(smem, S, jlo, jhi, jj, XH, YH, ZH, SC,
                                                                      P.pscale, iv, vv, st.n_eval, st.n_rck);
                        else
                            sweep_rppi32_pp<I, PP, true, EVALS, false>(smem, S, jlo, jhi, jj, XH, YH, ZH, SC,
                                                                       P.pscale, iv, vv, st.n_eval, st.n_rck);
                    } else {
                        if (S.lin)
                            sweep_rppi32_pp<I, PP, false, EVALS, true>(smem, S, jlo, jhi, jj, XH, YH, ZH, SC,
                                                                       P.pscale, iv, vv, st.n_eval, st.n_rck);
                        else
                            sweep_rppi32_pp<I, PP, false, EVALS, false>(smem, S, jlo, jhi, jj, XH, YH, ZH, SC,
                                                                        P.pscale, iv, vv, st.n_eval, st.n_rck);
                    }
                }
                if (pending > flush_at) {  // keep every shared u32 count far from overflow
                    __syncwarp();
                    flush_rppi(hc, nb, npi, P.hist, lane);
                    pending = 0;
                }
            }
        }
        return true;
    }
};

// Binary64 DD(rp, pi): canonical rp^2 and |dz|, exact edge compares.
template <int I, bool EVALS, bool WACC>
struct Rppi64Path {
    static __device__ __forceinline__ void init(const PairParams &P, unsigned char *smem)
    {
        const int nb = P.nbins, npi = P.npibins, row = npi + 1, copy = (nb + 1) * row;
        const Smem64 L = smem64_layout(P.tile_max, nb, npi, 0);
        double *E2 = reinterpret_cast<double *>(smem + L.e2);
        double *Pe = reinterpret_cast<double *>(smem + L.p);
        uint32_t *hist = reinterpret_cast<uint32_t *>(smem + P.hist_off);
        double *acc = WACC ? reinterpret_cast<double *>(smem + P.acc_off) : nullptr;

        const int tid = threadIdx.x;
        for (int q = tid; q <= nb; q += THREADS)
            E2[q] = P.E2[q];
        for (int q = tid; q <= npi; q += THREADS)
            Pe[q] = P.P[q];
        for (int q = tid; q < P.hcopies * copy; q += THREADS)
            hist[q] = 0u;
        if (WACC)
            for (int q = tid; q < 2 * P.hcopies * copy; q += THREADS)
                acc[q] = 0.0;
    }

    static __device__ __forceinline__ bool item(const PairParams &P, const Item &it,
                                                unsigned char *smem, PathState &st)
    {
        constexpr int J = 32 / I;
        const int nb = P.nbins, npi = P.npibins, row = npi + 1, copy = (nb + 1) * row;
        const Smem64 L = smem64_layout(P.tile_max, nb, npi, 0);
        uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
        double4_32a *tile = reinterpret_cast<double4_32a *>(smem + L.tile);
        double *E2 = reinterpret_cast<double *>(smem + L.e2);
        double *Pe = reinterpret_cast<double *>(smem + L.p);
        uint32_t *hist = reinterpret_cast<uint32_t *>(smem + P.hist_off);
        double *acc = WACC ? reinterpret_cast<double *>(smem + P.acc_off) : nullptr;

        const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
        unsigned &phase = st.phase;
        u64 &n_eval = st.n_eval;
        unsigned &pending = st.pending;

        uint32_t *hc = hist + (warp % P.hcopies) * copy;
        double *ac = WACC ? acc + 2 * (warp % P.hcopies) * copy : nullptr;
        const unsigned flush_at = (1u << 30) / (unsigned)(WARPS / P.hcopies);
        const int ii = lane % I, jj = lane / I;
        const double qnan = __longlong_as_double(0x7ff8000000000000ll);

        const double dzw = __dadd_rn(it.dzmax, 1e-9 * (P.rz + P.g.box[2] + 1.0));
        const int nchunks = (it.a1 - it.a0 + I - 1) / I;

        for (int t0 = it.b0; t0 < it.b1; t0 += P.tile_max) {
            const int nt = min(P.tile_max, it.b1 - t0);
            if (!stage_tile(tile, P.B.pos64 + t0, nt, 32, bar, phase, P.err, P.wait_ns)) {
                return false;
            }
            double zt_hi = tile[nt - 1].z;
            if (isnan(zt_hi))
                zt_hi = INFINITY;
            const double zt_lo = tile[0].z;
            auto zkey = [&](int p) { return tile[p].z; };
            auto next_chunk = [&]() {  // chunks in increasing order, claimed by the warps
                int v = 0;
                if (lane == 0)
                    v = atomicAdd(reinterpret_cast<int *>(smem + CLAIM_OFF), 1);
                return __shfl_sync(FULL, v, 0);
            };
            for (int c = next_chunk(); c < nchunks; c = next_chunk()) {
                const int ib = it.a0 + c * I;
                const int nvi = min(I, it.a1 - ib);
                const int i = ib + ii;
                const bool vi = ii < nvi;
                double4_32a pi = make_double4_32a(qnan, qnan, qnan, qnan);
                if (vi)
                    pi = P.A.pos64[i];
                const double zlo = __shfl_sync(FULL, pi.z, 0);
                double zhi = pi.z;
    #pragma unroll
                for (int o = 1; o < I; o <<= 1) {
                    const double t = __shfl_xor_sync(FULL, zhi, o);
                    zhi = (isnan(zhi) || t > zhi) ? t : zhi;
                }
                if (isnan(zlo))
                    continue;
                for (int k = it.kmin; k <= it.kmax; ++k) {
                    const double kz = k * P.g.box[2];
                    const double wlo = zlo - kz - dzw, whi = zhi - kz + dzw;
                    if (whi < zt_lo || wlo > zt_hi)
                        continue;
                    int jlo = warp_bound(zkey, nt, wlo, false, lane);
                    const int jhi = warp_bound(zkey, nt, whi, true, lane);
                    const bool tri = it.self && k == 0;
                    if (tri)
                        jlo = max(jlo, ib + 1 - t0);
                    if (jlo >= jhi)
                        continue;
                    pending += (unsigned)((jhi - jlo + J - 1) / J) * 32u;
                    const bool noshift = it.Sx == 0.0 && it.Sy == 0.0 && kz == 0.0;  // as in Xi64Path
                    for (int jb = jlo; jb < jhi; jb += J) {
                        const int j = jb + jj;
                        const double4_32a pj = tile[j];
                        const bool live = !tri || (t0 + j > i);
                        if (EVALS)
                            n_eval += (vi && j < jhi && live) ? 1ull : 0ull;
                        double dx, dy, dz;
                        if (noshift) {
                            dx = __dsub_rn(pj.x, pi.x);
                            dy = __dsub_rn(pj.y, pi.y);
                            dz = __dsub_rn(pj.z, pi.z);
                        } else {
                            dx = canon_comp(pi.x, pj.x, it.Sx);
                            dy = canon_comp(pi.y, pj.y, it.Sy);
                            dz = canon_comp(pi.z, pj.z, kz);
                        }
                        double rp2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
                        if (!live)
                            rp2 = qnan;
                        const int kb = bin_f64(rp2, E2, nb);
                        if (kb >= 0) {
                            const int m = bin_f64(fabs(dz), Pe, npi);
                            if (m >= 0) {
                                atomicAdd(&hc[kb * row + m], 1u);
                                if (WACC) {  // Code 1's weight; the oracle's product and sqrt
                                    const double pw = P.weighted ? __dmul_rn(pi.w, pj.w) : 1.0;
                                    atomicAdd(ac + 2 * (kb * row + m), pw);
                                    if (P.want_r)
                                        atomicAdd(ac + 2 * (kb * row + m) + 1,
                                                  __dmul_rn(__dsqrt_rn(rp2), pw));
                                }
                            }
                        }
                    }
                }
                if (pending > flush_at) {
                    __syncwarp();
                    flush_rppi(hc, nb, npi, P.hist, lane);
                    pending = 0;
                }
            }
        }
        return true;
    }

    static __device__ __forceinline__ void fini(const PairParams &P, unsigned char *smem, PathState &st)
    {
        uint32_t *hist = reinterpret_cast<uint32_t *>(smem + P.hist_off);
        double *acc = WACC ? reinterpret_cast<double *>(smem + P.acc_off) : nullptr;

        const int tid = threadIdx.x, lane = tid & 31;
        u64 &n_eval = st.n_eval;

        __syncthreads();
        merge_rppi(P, hist, acc, P.nbins + 1);
        n_eval = warp_sum_u64(n_eval);
        if (lane == 0 && n_eval)
            atomicAdd(&P.diag[1], n_eval);
    }
};

// One persistent kernel per path: init the CTA's tables and histograms, pull
// kept column pairs from the global counter, merge at the end.
template <class Path, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_path(const __grid_constant__ PairParams P)
{
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    volatile int *s_item = reinterpret_cast<volatile int *>(smem + 8);
    Path::init(P, smem);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    PathState st = {0ull, 0ull, 0ull, 0u, 0u, 0u};
    const int n_work = (int)*P.work_count;
    for (;;) {
        if (threadIdx.x == 0)
            *s_item = (int)atomicAdd(P.item_counter, 1u);
        __syncthreads();
        const int item = *s_item;
        __syncthreads();
        if (item >= n_work)
            break;
        Item it;
        decode_item(P, item, it);
        if (!Path::item(P, it, smem, st))
            break;
    }
    __syncthreads();
    Path::fini(P, smem, st);
}

// ============================================ pipelined float32 DD(r) kernel
// Two tile buffers: while the warps sweep the tile in one, the next tile is
// already staged in the other, so no CTA-wide barrier separates work items.
// A unit is one tile of one work item.  The warp that finishes a unit last
// (counted in done[s]) refills its buffer with the unit after next: it claims
// the next item when the cursor's item has no tile left, pads, and issues the
// bulk copies; the other warps move straight on to the other buffer.  Within
// a unit the warps claim chunks from claim[s].  Every wait is bounded.
struct PipeHdr {
    uint64_t full[2];    // tile-ready barrier of each buffer
    WorkItem w[2];       // work item of each buffer's unit
    int item[2];         // its index (-1: no more work)
    int t0[2], nt[2];    // its tile of column b
    int claim[2];        // next chunk of the unit
    int done[2];         // warps finished with the unit
    int cur, next_t0;    // cursor: item of the last issued unit, start of its next tile
};
static_assert(sizeof(PipeHdr) <= XI32_LUT_OFF, "pipeline header fits before the table");

// Fill buffer s with the next unit (called by one whole warp; lane 0 claims,
// every lane pads, lane 0 issues the copies and arrives on the barrier).
__device__ __forceinline__ void pipe_issue(const PairParams &P, PipeHdr *H, int s, int n_work,
                                           unsigned char *buf, int lane, bool stall = false)
{
    int item = -1, t0 = 0, nt = 0;
    if (lane == 0) {
        const int cur = H->cur;
        if (cur >= 0 && H->next_t0 < H->w[s ^ 1].b1 && H->item[s ^ 1] == cur) {
            item = cur;  // the cursor's item has tiles left (its record is in the other buffer)
            t0 = H->next_t0;
            H->w[s] = H->w[s ^ 1];
        } else {
            for (;;) {  // next item with points on both sides (bounded by the work count)
                const int c = (int)atomicAdd(P.item_counter, 1u);
                if (c >= n_work)
                    break;
                const WorkItem w = P.work[c];
                if (w.a1 > w.a0 && w.b1 > w.b0) {
                    item = c;
                    t0 = w.b0;
                    H->w[s] = w;
                    break;
                }
            }
            H->cur = item;
        }
        if (item >= 0) {
            nt = min(TILE32, H->w[s].b1 - t0);
            H->next_t0 = t0 + nt;
        }
    }
    item = __shfl_sync(FULL, item, 0);
    nt = __shfl_sync(FULL, nt, 0);
    t0 = __shfl_sync(FULL, t0, 0);
    if (item >= 0) {
        float *t = reinterpret_cast<float *>(buf);
        for (int q = lane; q < 3 * 64; q += 32)  // sentinels after the copied range: never counted
            t[(q >> 6) * (XI32_TSTRIDE / 4) + nt + (q & 63)] = __int_as_float(0x7fc00000);
    }
    __syncwarp();
    if (lane == 0) {
        H->item[s] = item;
        H->t0[s] = t0;
        H->nt[s] = nt;
        if (item >= 0) {
            const unsigned bytes = (unsigned)nt * 4u;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&H->full[s], 3u * bytes);
            if (!stall) {  // diagnostic stall: the armed copy is never issued
                bulk_g2s(buf, P.B.xs + t0, bytes, &H->full[s]);
                bulk_g2s(buf + XI32_TSTRIDE, P.B.ys + t0, bytes, &H->full[s]);
                bulk_g2s(buf + 2 * XI32_TSTRIDE, P.B.zs + t0, bytes, &H->full[s]);
            }
        } else {
            mbar_arrive(&H->full[s]);
        }
    }
}

template <class Path, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_pipe(const __grid_constant__ PairParams P)
{
    extern __shared__ __align__(128) unsigned char smem[];
    PipeHdr *H = reinterpret_cast<PipeHdr *>(smem);
    unsigned char *buf0 = smem + XI32_TX_OFF, *buf1 = smem + pipe_slot1_off(P.nbins);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Path::init(P, smem);
    if (threadIdx.x == 0) {
        mbar_init(&H->full[0], 1);
        mbar_init(&H->full[1], 1);
        fence_mbar_init();
        H->item[0] = H->item[1] = -1;
        H->claim[0] = H->claim[1] = 0;
        H->done[0] = H->done[1] = 0;
        H->cur = -1;
        H->next_t0 = 0;
    }
    __syncthreads();
    const int n_work = (int)*P.work_count;
    if (warp == 0) {
        pipe_issue(P, H, 0, n_work, buf0, lane, (P.flags & CF_FLAG_DEBUG_STALL) != 0);
        pipe_issue(P, H, 1, n_work, buf1, lane);
    }
    PathState st = {0ull, 0ull, 0ull, 0u, 0u, 0u};
    unsigned par = 0u;  // bit s: parity of buffer s's next phase
    bool timed_out = false;
    for (int u = 0;; ++u) {
        const int s = u & 1;
        unsigned char *buf = s ? buf1 : buf0;
        if (!mbar_wait(&H->full[s], (par >> s) & 1u, P.wait_ns)) {
            if (lane == 0)
                atomicOr(P.err, ERR_TIMEOUT);
            timed_out = true;
            break;
        }
        par ^= 1u << s;
        const int item = reinterpret_cast<volatile int *>(H->item)[s];
        if (item < 0)
            break;
        Item it;
        decode_record(P, H->w[s], it);
        Path::tile(P, it, H->t0[s], H->nt[s], buf, &H->claim[s], smem, st);
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            __threadfence_block();  // this warp's reads of the buffer come first
            last = atomicAdd(&H->done[s], 1) == WARPS - 1;
        }
        if (__shfl_sync(FULL, last, 0)) {
            if (lane == 0) {
                __threadfence_block();
                H->done[s] = 0;
                H->claim[s] = 0;
            }
            __syncwarp();
            pipe_issue(P, H, s, n_work, buf, lane);
        }
    }
    if (__syncthreads_or(timed_out)) {
        // every warp gave up at the same unit: let the copies still in flight (the
        // other buffer's, and a late one of the stuck buffer) land before the CTA
        // exits, each wait bounded again
        if (threadIdx.x == 0) {
            mbar_wait(&H->full[0], par & 1u, P.wait_ns);
            mbar_wait(&H->full[1], (par >> 1) & 1u, P.wait_ns);
        }
        __syncthreads();
    }
    Path::fini(P, smem, st);
}

// ============================================================ batched kernel
// Many independent jobs (catalogues, bins, modes) in one persistent launch: the
// CTAs pull items from one global counter over the concatenation of the jobs'
// kept column pairs; a CTA that moves on to another job merges its histograms
// into the previous job's output and loads the next job's tables.
using XiF32 = Xi32Path<16, 2, false, false>;
using XiF32_8x2 = Xi32Path<8, 2, false, false>;
using XiF32_16x1 = Xi32Path<16, 1, false, false>;
using XiF32_32x1 = Xi32Path<32, 1, false, false>;
using XiF64 = Xi64Path<8, false, false>;
using RpF32 = Rppi32PathPP<16, 2, false>;
using RpF64 = Rppi64Path<8, false, false>;

__device__ __forceinline__ void batch_init(int path, const PairParams &P, unsigned char *smem)
{
    switch (path) {
    case BATCH_XI32:
    case BATCH_XI32_8x2:
    case BATCH_XI32_16x1:
    case BATCH_XI32_32x1: XiF32::init(P, smem); break;  // shape-independent
    case BATCH_XI64: XiF64::init(P, smem); break;
    case BATCH_RPPI32: RpF32::init(P, smem); break;
    default: RpF64::init(P, smem); break;
    }
}

__device__ __forceinline__ bool batch_item(int path, const PairParams &P, const Item &it,
                                           unsigned char *smem, PathState &st)
{
    switch (path) {
    case BATCH_XI32: return XiF32::item(P, it, smem, st);
    case BATCH_XI32_8x2: return XiF32_8x2::item(P, it, smem, st);
    case BATCH_XI32_16x1: return XiF32_16x1::item(P, it, smem, st);
    case BATCH_XI32_32x1: return XiF32_32x1::item(P, it, smem, st);
    case BATCH_XI64: return XiF64::item(P, it, smem, st);
    case BATCH_RPPI32: return RpF32::item(P, it, smem, st);
    default: return RpF64::item(P, it, smem, st);
    }
}

__device__ __forceinline__ void batch_fini(int path, const PairParams &P, unsigned char *smem,
                                           PathState &st)
{
    switch (path) {
    case BATCH_XI32:
    case BATCH_XI32_8x2:
    case BATCH_XI32_16x1:
    case BATCH_XI32_32x1: XiF32::fini(P, smem, st); break;  // shape-independent
    case BATCH_XI64: XiF64::fini(P, smem, st); break;
    case BATCH_RPPI32: RpF32::fini(P, smem, st); break;
    default: RpF64::fini(P, smem, st); break;
    }
}

// offsets[j] = kept column pairs of jobs 0..j-1 (one thread; a few thousand jobs at most).
// Exclusive scan of the jobs' kept-item counts (one warp: each lane loads its
// jobs' counts in parallel, 32 jobs per round).
__global__ void k_batch_offsets(const __grid_constant__ BatchParams B)
{
    if (blockIdx.x != 0)
        return;
    const int lane = threadIdx.x & 31;
    unsigned carry = 0;
    for (int j0 = 0; j0 < B.njobs; j0 += 32) {
        const int j = j0 + lane;
        const unsigned v = j < B.njobs ? *B.jobs[j].work_count : 0u;
        unsigned incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o)
                incl += t;
        }
        if (j < B.njobs)
            B.offsets[j] = carry + incl - v;
        carry += __shfl_sync(FULL, incl, 31);
    }
    if (lane == 0)
        B.offsets[B.njobs] = carry;
}

// Candidate pairs of a work item below which the batch kernel claims items in
// groups (see k_batch).
constexpr long long GROUP_PAIRS = 1ll << 16;

__global__ void __launch_bounds__(THREADS, 2) k_batch(const __grid_constant__ BatchParams B)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned s_off[BATCH_MAX + 1];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    volatile int *s_item = reinterpret_cast<volatile int *>(smem + 8);
    for (int j = threadIdx.x; j <= B.njobs; j += THREADS)
        s_off[j] = B.offsets[j];
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const unsigned total = s_off[B.njobs];
    // Small items (column pairs of fewer than GROUP_PAIRS candidate pairs) are
    // claimed in groups of consecutive items (up to 16, together about
    // GROUP_PAIRS), so that a CTA stays on a small job for a while instead of
    // every CTA switching to it for one item (each switch loads the job's table
    // and merges its histogram); larger items are claimed one by one, which keeps
    // the load balanced.  The size of the next group comes from the last item
    // decoded (the next one is most often of the same job), so a claim stays one
    // atomic.
    PathState st = {0ull, 0ull, 0ull, 0u, 0u, 0u};
    int cur = -1;
    unsigned group = 1;
    bool ok = true;
    while (ok) {
        if (threadIdx.x == 0)
            *s_item = (int)atomicAdd(B.item_counter, group);
        __syncthreads();
        const unsigned base = (unsigned)*s_item;
        __syncthreads();
        if (base >= total)
            break;
        const unsigned stop = min(base + group, total);
#pragma unroll 1
        for (unsigned item = base; item < stop; ++item) {
            int lo = 0, hi = B.njobs;  // largest job with s_off[job] <= item
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_off[mid] <= item)
                    lo = mid;
                else
                    hi = mid;
            }
            const int job = lo;
            if (job != cur) {  // CTA-uniform: every thread holds the same item
                if (cur >= 0)
                    batch_fini(B.path[cur], B.jobs[cur], smem, st);
                __syncthreads();
                batch_init(B.path[job], B.jobs[job], smem);
                st.n_eval = st.n_rck = st.n_viol = 0ull;
                st.pending = 0u;
                __syncthreads();
                cur = job;
            }
            const PairParams &P = B.jobs[job];
            Item it;
            decode_item(P, (int)(item - s_off[job]), it);
            const long long pairs = (long long)max(it.a1 - it.a0, 1) * max(it.b1 - it.b0, 1);
            group = pairs < GROUP_PAIRS ? (unsigned)min(16ll, GROUP_PAIRS / pairs) : 1u;
            if (!batch_item(B.path[job], P, it, smem, st)) {
                ok = false;
                break;
            }
        }
    }
    if (cur >= 0)
        batch_fini(B.path[cur], B.jobs[cur], smem, st);
}

// Per (kernel, device): the dynamic shared-memory limit set so far (only ever
// raised) and the occupancy per shared-memory size, queried once.
struct OccCache {
    const void *kern;
    int dev, smem, occ;
};
struct AttrCache {
    const void *kern;
    int dev, limit;
};
OccCache g_occ[128];
AttrCache g_attr[32];
int g_nocc = 0, g_nattr = 0;
std::mutex g_occ_mu;

template <class K>
cudaError_t occupancy(K kern, int smem, int &occ)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e)
        return e;
    std::lock_guard<std::mutex> lock(g_occ_mu);
    AttrCache *a = nullptr;
    for (int q = 0; q < g_nattr; ++q)
        if (g_attr[q].kern == (const void *)kern && g_attr[q].dev == dev)
            a = &g_attr[q];
    if (!a || a->limit < smem) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e)
            return e;
        if (!a && g_nattr < 32)
            a = &g_attr[g_nattr++];
        if (a)
            *a = AttrCache{(const void *)kern, dev, smem};
    }
    for (int q = 0; q < g_nocc; ++q)
        if (g_occ[q].kern == (const void *)kern && g_occ[q].dev == dev && g_occ[q].smem == smem) {
            occ = g_occ[q].occ;
            return cudaSuccess;
        }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, THREADS, smem);
    if (e)
        return e;
    if (g_nocc < 128)
        g_occ[g_nocc++] = OccCache{(const void *)kern, dev, smem, occ};
    return cudaSuccess;
}

template <class K>
cudaError_t launch_persistent(K kern, const PairParams &P, PairLaunch &L, int sms, cudaStream_t st)
{
    int occ = 0;
    cudaError_t e = occupancy(kern, L.smem, occ);
    if (e)
        return e;
    if (occ < 1)
        return cudaErrorInvalidConfiguration;
    long long blocks = (long long)sms * occ;
    if (L.max_blocks > 0 && blocks > L.max_blocks)
        blocks = L.max_blocks;  // per-CTA scratch was sized for this many
    if (blocks > P.n_items)
        blocks = P.n_items > 0 ? P.n_items : 1;
    L.blocks = (int)blocks;
    kern<<<L.blocks, THREADS, L.smem, st>>>(P);
    return cudaGetLastError();
}

}  // namespace

int batch_path(const PairParams &P, int f64, int chunk, int pp)
{
    if (P.kind == 0) {
        if (f64)
            return BATCH_XI64;
        if (pp == 2 && chunk == 8)
            return BATCH_XI32_8x2;
        if (pp == 1 && chunk == 16)
            return BATCH_XI32_16x1;
        if (pp == 1 && chunk == 32)
            return BATCH_XI32_32x1;
        return BATCH_XI32;
    }
    return f64 ? BATCH_RPPI64 : BATCH_RPPI32;
}

cudaError_t launch_worklist(const PairParams &P, cudaStream_t st)
{
    if (P.n_items <= 0)
        return cudaSuccess;
    k_worklist<<<(P.n_items + 255) / 256, 256, 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_worklist_batch(const PairParams *jobs, const unsigned *pre, int njobs,
                                  unsigned blocks, cudaStream_t st)
{
    if (blocks == 0 || njobs < 1)
        return cudaSuccess;
    k_worklist_batch<<<blocks, 256, 0, st>>>(jobs, pre, njobs);
    return cudaGetLastError();
}

cudaError_t launch_batch(const BatchParams &B, int smem, int sms, int &blocks, cudaStream_t st)
{
    if (B.njobs < 1 || B.njobs > BATCH_MAX)
        return cudaErrorInvalidValue;
    k_batch_offsets<<<1, 32, 0, st>>>(B);
    cudaError_t e = cudaGetLastError();
    if (e)
        return e;
    int occ = 0;
    if ((e = occupancy(k_batch, smem, occ)))
        return e;
    if (occ < 1)
        return cudaErrorInvalidConfiguration;
    blocks = sms * occ;
    k_batch<<<blocks, THREADS, smem, st>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_pairs(const PairParams &P0, PairLaunch &L, int sms, cudaStream_t st)
{
    L.kernels = 0;
    if (P0.n_items <= 0)
        return cudaSuccess;
    PairParams P = P0;
    // the float32 DD(r) kernels take their chunk windows from the window pre-pass
    const bool xi32 = P.kind == 0 && !L.f64;
    if (xi32 && !P.win)
        return cudaErrorInvalidValue;  // the caller provides the window records
    P.win_chunk = xi32 ? xi32_chunk(L.chunk, L.pp, P.wacc != 0, L.verify != 0) : 0;
    k_worklist<<<(P.n_items + 255) / 256, 256, 0, st>>>(P);
    cudaError_t e = cudaGetLastError();
    if (e)
        return e;
    L.kernels = 2;
    if (xi32) {
        const int wblocks = std::max(1, std::min((P.n_items + 3) / 4, sms * 16));
        k_windows<<<wblocks, 128, 0, st>>>(P);
        if ((e = cudaGetLastError()))
            return e;
        L.kernels = 3;
    }
    if (P.kind == 1) {
        if (L.f64) {
            if (P.wacc)
                return L.evals ? launch_persistent(k_path<Rppi64Path<8, true, true>, 1>, P, L, sms, st)
                               : launch_persistent(k_path<Rppi64Path<8, false, true>, 1>, P, L, sms, st);
            return L.evals ? launch_persistent(k_path<Rppi64Path<8, true, false>, 1>, P, L, sms, st)
                           : launch_persistent(k_path<Rppi64Path<8, false, false>, 1>, P, L, sms, st);
        }
        if (P.wacc)
            return L.evals ? launch_persistent(k_path<Rppi32Path<16, true, false, true>, 3>, P, L, sms, st)
                           : launch_persistent(k_path<Rppi32Path<16, false, false, true>, 3>, P, L, sms, st);
        if (L.verify)
            return launch_persistent(k_path<Rppi32Path<8, true, true, false>, 3>, P, L, sms, st);
        if (L.pp == 2)  // two primaries per lane, deferred flags
            return L.evals ? launch_persistent(k_path<Rppi32PathPP<16, 2, true>, 3>, P, L, sms, st)
                           : launch_persistent(k_path<Rppi32PathPP<16, 2, false>, 3>, P, L, sms, st);
        switch (L.chunk) {
        case 16:
            return L.evals ? launch_persistent(k_path<Rppi32Path<16, true, false, false>, 3>, P, L, sms, st)
                           : launch_persistent(k_path<Rppi32Path<16, false, false, false>, 3>, P, L, sms, st);
        case 32:
            return L.evals ? launch_persistent(k_path<Rppi32Path<32, true, false, false>, 3>, P, L, sms, st)
                           : launch_persistent(k_path<Rppi32Path<32, false, false, false>, 3>, P, L, sms, st);
        default:
            return L.evals ? launch_persistent(k_path<Rppi32Path<8, true, false, false>, 3>, P, L, sms, st)
                           : launch_persistent(k_path<Rppi32Path<8, false, false, false>, 3>, P, L, sms, st);
        }
    }
    if (P.kind != 0)
        return cudaErrorNotSupported;
    if (L.f64) {
        if (P.wacc)
            return L.evals ? launch_persistent(k_path<Xi64Path<8, true, true>, 1>, P, L, sms, st)
                           : launch_persistent(k_path<Xi64Path<8, false, true>, 1>, P, L, sms, st);
        return L.evals ? launch_persistent(k_path<Xi64Path<8, true, false>, 1>, P, L, sms, st)
                       : launch_persistent(k_path<Xi64Path<8, false, false>, 1>, P, L, sms, st);
    }
    constexpr int HW = WARPS;
    constexpr bool PW = true;
    if (P.wacc) {  // pair weights and / or mean separation: integer sums in the same sweep
        if (P.want_r && P.rlo) {  // r from residual-corrected squared distances
            if (P.weighted)
                return L.evals ? launch_persistent(k_path<Xi32Path<16, 1, true, false, true, true, HW, PW, -1, true>, 2>, P, L, sms, st)
                               : launch_persistent(k_path<Xi32Path<16, 1, false, false, true, true, HW, PW, -1, true>, 2>, P, L, sms, st);
            return L.evals ? launch_persistent(k_path<Xi32Path<16, 1, true, false, false, true, HW, PW, -1, true>, 2>, P, L, sms, st)
                           : launch_persistent(k_path<Xi32Path<16, 1, false, false, false, true, HW, PW, -1, true>, 2>, P, L, sms, st);
        }
        if (P.weighted && P.want_r)
            return L.evals ? launch_persistent(k_path<Xi32Path<16, 1, true, false, true, true, HW, PW>, 2>, P, L, sms, st)
                           : launch_persistent(k_path<Xi32Path<16, 1, false, false, true, true, HW, PW>, 2>, P, L, sms, st);
        if (P.weighted)
            return L.evals ? launch_persistent(k_path<Xi32Path<16, 1, true, false, true, false, HW, PW>, 2>, P, L, sms, st)
                           : launch_persistent(k_path<Xi32Path<16, 1, false, false, true, false, HW, PW>, 2>, P, L, sms, st);
        return L.evals ? launch_persistent(k_path<Xi32Path<16, 1, true, false, false, true, HW, PW>, 2>, P, L, sms, st)
                       : launch_persistent(k_path<Xi32Path<16, 1, false, false, false, true, HW, PW>, 2>, P, L, sms, st);
    }
    if (!L.pipe) {  // single tile buffer, one histogram copy per warp
        if (L.verify)
            return launch_persistent(k_path<Xi32Path<8, 1, true, true, false, false, HW, PW>, 3>, P, L, sms, st);
        return L.evals ? launch_persistent(k_path<Xi32Path<16, 2, true, false, false, false, HW, PW>, 3>, P, L, sms, st)
                       : launch_persistent(k_path<Xi32Path<16, 2, false, false, false, false, HW, PW>, 3>, P, L, sms, st);
    }
    // two tile buffers, one shared histogram copy
    constexpr int H1 = 1;
    if (L.verify)
        return launch_persistent(k_pipe<Xi32Path<8, 1, true, true, false, false, H1, PW>, 3>, P, L, sms, st);
    if (L.pp == 4)
        return L.evals ? launch_persistent(k_pipe<Xi32Path<8, 4, true, false, false, false, H1, PW>, 2>, P, L, sms, st)
                       : launch_persistent(k_pipe<Xi32Path<8, 4, false, false, false, false, H1, PW>, 2>, P, L, sms, st);
    if (L.pp == 2) {
        if (L.chunk == 8)
            return L.evals ? launch_persistent(k_pipe<Xi32Path<8, 2, true, false, false, false, H1, PW>, 3>, P, L, sms, st)
                           : launch_persistent(k_pipe<Xi32Path<8, 2, false, false, false, false, H1, PW>, 3>, P, L, sms, st);
        return L.evals ? launch_persistent(k_pipe<Xi32Path<16, 2, true, false, false, false, H1, PW>, 3>, P, L, sms, st)
                       : launch_persistent(k_pipe<Xi32Path<16, 2, false, false, false, false, H1, PW>, 3>, P, L, sms, st);
    }
    switch (L.chunk) {
    case 16:
        return L.evals ? launch_persistent(k_pipe<Xi32Path<16, 1, true, false, false, false, H1, PW>, 3>, P, L, sms, st)
                       : launch_persistent(k_pipe<Xi32Path<16, 1, false, false, false, false, H1, PW>, 3>, P, L, sms, st);
    case 32:
        return L.evals ? launch_persistent(k_pipe<Xi32Path<32, 1, true, false, false, false, H1, PW>, 3>, P, L, sms, st)
                       : launch_persistent(k_pipe<Xi32Path<32, 1, false, false, false, false, H1, PW>, 3>, P, L, sms, st);
    default:
        return L.evals ? launch_persistent(k_pipe<Xi32Path<8, 1, true, false, false, false, H1, PW>, 3>, P, L, sms, st)
                       : launch_persistent(k_pipe<Xi32Path<8, 1, false, false, false, false, H1, PW>, 3>, P, L, sms, st);
    }
}

}  // namespace cf
