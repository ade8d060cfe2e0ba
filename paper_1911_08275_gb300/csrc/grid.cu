// GPU gridding (Sec. 1.2 and 2.1 of arXiv:1911.08275): points are binned into
// columns of side >= Rmax / refine in x and y, each column is sorted along z
// (the paper's z-sort that shrinks the search window from 3*pimax to 2*pimax),
// and each column gets its (x, y) bounding box for the pruning of Sec. 2.2.
//
// Layout produced (one gridded catalogue):
//   cell_start[ncells + 1]  counting-sort offsets; cell = column * nz + zcell,
//                           column = cx * ncy + cy.  A column is the contiguous
//                           range [cell_start[col*nz], cell_start[(col+1)*nz]),
//                           padded at its end to a multiple of 4 entries (16 bytes
//                           of float) so 1-D bulk copies of column slices are
//                           aligned; padding entries are NaN and never counted.
//   xs, ys, zs[n']  float32 x - ox, y - oy, z - oz (grid frame), structure of arrays
//   pos64[n']       double4 (x, y, z, w) exact binary64 copies (re-checks, FP64 path)
//   perm[n']        original index of each sorted point (-1 for padding)
//   colbox[ncols]   (xmin, xmax, ymin, ymax) of the column's points, binary64
// with n' <= n + 3 * ncols.
//
// Within a cell the order is (z, original index), computed by ranking, so the
// output is deterministic whatever the order of the atomic slot assignment.
#include <cuda_runtime.h>
#include <float.h>

#include <algorithm>

#include "cf_internal.cuh"
#include "grid.cuh"

namespace cf {

namespace {

// Order-preserving map of a binary64 bit pattern onto uint64 (and back).
__device__ __forceinline__ unsigned long long order_key(long long b)
{
    const unsigned long long u = (unsigned long long)b;
    return (b < 0) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_value(unsigned long long k)
{
    const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}


// Validity and float32 frame coordinate of one input coordinate, without
// binary64 arithmetic (the binary64 pipe of this GPU is narrow): range tests on
// bit patterns, one conversion.
__device__ __forceinline__ bool coord(double v, int a, const Geom &g, float &f)
{
    const long long b = __double_as_longlong(v);
    if (g.periodic) {
        f = __double2float_rn(v);  // frame origin is 0
        return (b >= 0 && b < g.box_bits[a]) || b == (long long)0x8000000000000000ull;
    }
    f = __double2float_rn(__dsub_rn(v, g.origin[a]));
    return (b & 0x7ff0000000000000ll) != 0x7ff0000000000000ll;
}
__device__ __forceinline__ bool coord(float v, int a, const Geom &g, float &f)
{
    const int b = __float_as_int(v);
    if (g.periodic) {
        f = v;
        return (b >= 0 && b < g.box_bits32[a]) || b == (int)0x80000000u;
    }
    f = __double2float_rn(__dsub_rn((double)v, g.origin[a]));
    return (b & 0x7f800000) != 0x7f800000;
}

template <class T>
__global__ void k_assign(const T *__restrict__ x, const T *__restrict__ y, const T *__restrict__ z,
                         long long n, Geom g, uint32_t *__restrict__ cell_of,
                         uint32_t *__restrict__ slot, uint32_t *__restrict__ count,
                         unsigned *__restrict__ err)
{
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // every lane of a warp runs the same number of iterations (warp-wide match)
    const long long first = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    for (long long base = first; base < n; base += stride) {
        const long long p = base + lane;
        const bool live = p < n;
        uint32_t cell = 0xffffffffu;
        if (live) {
            float fx, fy, fz;
            const bool ok = coord(x[p], 0, g, fx) & coord(y[p], 1, g, fy) & coord(z[p], 2, g, fz);
            if (!ok) {
                atomicOr(err, ERR_COORD);
                fx = fy = fz = 0.0f;
            }
            const int cx = cell_index_f(fx, g.inv_wf[0], g.ncx);
            const int cy = cell_index_f(fy, g.inv_wf[1], g.ncy);
            const int cz = cell_index_f(fz, g.inv_wf[2], g.nz);
            cell = (uint32_t)(((long long)(cx * g.ncy + cy)) * g.nz + cz);
        }
        // clustered inputs put runs of points into one cell: one atomic per group
        const unsigned same = __match_any_sync(FULL, cell);
        const int leader = __ffs(same) - 1;
        uint32_t b0 = 0;
        if (live && lane == leader)
            b0 = atomicAdd(&count[cell], (uint32_t)__popc(same));
        b0 = __shfl_sync(FULL, b0, leader);
        if (live) {
            cell_of[p] = cell;
            slot[p] = b0 + (uint32_t)__popc(same & ((1u << lane) - 1u));
        }
    }
}

// Exclusive scan, 3 phases: per-block scan of SCAN_ITEMS elements, scan of the
// block sums (one block), add-back.
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_PER_THREAD = 4;
constexpr int SCAN_ITEMS = SCAN_THREADS * SCAN_PER_THREAD;

__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_sums, uint32_t *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o)
            incl += t;
    }
    if (lane == 31)
        warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t s = lane < nw ? warp_sums[lane] : 0u;
        uint32_t si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(FULL, si, o);
            if (lane >= o)
                si += t;
        }
        if (lane < nw)
            warp_sums[lane] = si - s;
        if (lane == 31)
            *total = si;
    }
    __syncthreads();
    const uint32_t r = warp_sums[wid] + incl - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAN_THREADS)
    k_scan_blocks(const uint32_t *in, uint32_t *out, long long n, uint32_t *__restrict__ bsum)
{
    __shared__ uint32_t ws[32];
    __shared__ uint32_t tot;
    const long long base = (long long)blockIdx.x * SCAN_ITEMS + threadIdx.x * SCAN_PER_THREAD;
    uint32_t v[SCAN_PER_THREAD];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0u;
        s += v[k];
    }
    uint32_t pre = block_exclusive_scan(s, ws, &tot);
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        if (base + k < n)
            out[base + k] = pre;
        pre += v[k];
    }
    if (threadIdx.x == 0)
        bsum[blockIdx.x] = tot;
}

// Exclusive scan of the block sums in place (one block, SCAN_ITEMS at a time
// with a running carry); *grand gets the total.
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_sums(uint32_t *bsum, long long nb, uint32_t *grand)
{
    __shared__ uint32_t ws[32];
    __shared__ uint32_t tot;
    uint32_t carry = 0;
    for (long long c = 0; c < nb; c += SCAN_ITEMS) {
        uint32_t v[SCAN_PER_THREAD];
        uint32_t s = 0;
        const long long base = c + threadIdx.x * SCAN_PER_THREAD;
#pragma unroll
        for (int k = 0; k < SCAN_PER_THREAD; ++k) {
            v[k] = (base + k < nb) ? bsum[base + k] : 0u;
            s += v[k];
        }
        uint32_t pre = carry + block_exclusive_scan(s, ws, &tot);
#pragma unroll
        for (int k = 0; k < SCAN_PER_THREAD; ++k) {
            if (base + k < nb)
                bsum[base + k] = pre;
            pre += v[k];
        }
        carry += tot;  // read before any thread can reach the next scan's write of tot
    }
    if (threadIdx.x == 0)
        *grand = carry;
}

__global__ void k_scan_add(uint32_t *__restrict__ out, long long n, const uint32_t *__restrict__ bsum)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        out[i] += bsum[i / SCAN_ITEMS];
}

// One warp per column: padding that rounds the column up to a multiple of 4,
// written into the padded count of the column's last cell.
__global__ void k_colpad(const uint32_t *__restrict__ count, int ncols, int nz,
                         uint32_t *__restrict__ pad, uint32_t *__restrict__ padded)
{
    const int lane = threadIdx.x & 31;
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (col >= ncols)
        return;
    const long long c0 = (long long)col * nz;
    uint32_t tot = 0;
    for (int z = lane; z < nz; z += 32) {
        const uint32_t v = count[c0 + z];
        padded[c0 + z] = v;
        tot += v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        tot += __shfl_xor_sync(FULL, tot, o);
    const uint32_t pd = (4u - (tot & 3u)) & 3u;
    __syncwarp();
    if (lane == 0) {
        pad[col] = pd;
        padded[c0 + nz - 1] += pd;
    }
}

template <class T>
__global__ void k_scatter(const T *__restrict__ z, long long n, const uint32_t *__restrict__ cell_of,
                          const uint32_t *__restrict__ slot, const uint32_t *__restrict__ start,
                          int *__restrict__ tmp_idx, unsigned long long *__restrict__ tmp_key)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const uint32_t q = start[cell_of[p]] + slot[p];
        tmp_idx[q] = (int)p;
        tmp_key[q] = order_key(__double_as_longlong((double)z[p]));
    }
}

// Write one ranked entry: binary64 copy, float32 frame coordinates, weight,
// original index.
template <class T>
__device__ __forceinline__ void put_entry(const T *__restrict__ x, const T *__restrict__ y,
                                          const double *__restrict__ w, const Geom &g, uint32_t d,
                                          int iq, unsigned long long kq, float *__restrict__ xs,
                                          float *__restrict__ ys, float *__restrict__ zs,
                                          float *__restrict__ ws, double4_32a *__restrict__ pos64,
                                          int *__restrict__ perm, unsigned &wm)
{
    const double X = (double)x[iq], Y = (double)y[iq], Z = key_value(kq);
    const double W = w ? w[iq] : 0.0;
    pos64[d] = make_double4_32a(X, Y, Z, W);
    float fx, fy, fz;
    coord(X, 0, g, fx);
    coord(Y, 1, g, fy);
    coord(Z, 2, g, fz);
    xs[d] = fx;
    ys[d] = fy;
    zs[d] = fz;
    if (ws) {
        ws[d] = (float)W;
        wm = max(wm, __float_as_uint(fabsf((float)W)));
    }
    perm[d] = iq;
}

constexpr int SORT_THREADS = 256;
constexpr int SORT_BUF = 256;  // entries of a cell ranked from shared memory

// Rank of entry (kq, iq) among the n entries of e[] by (key, original index).
__device__ __forceinline__ uint32_t rank_in(const ulonglong2 *e, uint32_t n, unsigned long long kq,
                                            int iq)
{
    uint32_t rank = 0;
    for (uint32_t m = 0; m < n; ++m) {
        const ulonglong2 em = e[m];  // every lane of the group reads the same entry
        rank += (em.x < kq) || (em.x == kq && (int)em.y < iq);
    }
    return rank;
}

// Rank the cells' real entries by (z, original index) and write the sorted
// float32 / binary64 copies.  Each warp claims two cells at a time from a
// counter (cell sizes vary, and a fixed split leaves a partial second wave of
// blocks): cells of up to 16 entries are ranked by a half warp each; otherwise
// the whole warp ranks the two cells one after the other, up to SORT_BUF
// entries, beyond that against the cell in global memory.  The entries being ranked are copied to a
// per-warp shared buffer as 16-byte (key, index) records: one broadcast load
// per comparison.
template <class T>
__global__ void __launch_bounds__(SORT_THREADS)
    k_sort_cells(const T *__restrict__ x, const T *__restrict__ y, const double *__restrict__ w,
                 long long ncells, Geom g, const uint32_t *__restrict__ count,
                 const uint32_t *__restrict__ start, const int *__restrict__ tmp_idx,
                 const unsigned long long *__restrict__ tmp_key, float *__restrict__ xs,
                 float *__restrict__ ys, float *__restrict__ zs, float *__restrict__ ws,
                 unsigned *__restrict__ wmax, double4_32a *__restrict__ pos64,
                 int *__restrict__ perm, unsigned *__restrict__ claim)
{
    __shared__ ulonglong2 s_ent[SORT_THREADS / 32][SORT_BUF];
    const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15, wid = threadIdx.x >> 5;
    ulonglong2 *be = s_ent[wid];
    unsigned wm = 0;  // bit pattern of the largest |w| (float) this thread stored
    for (;;) {
        unsigned v = 0u;
        if (lane == 0)
            v = atomicAdd(claim, 1u);  // the next pair of cells (zeroed with the counts)
        const long long c0 = 2ll * __shfl_sync(FULL, v, 0);
        if (c0 >= ncells)
            break;
        const long long cm = c0 + half;  // this half warp's cell
        const uint32_t cnt = cm < ncells ? count[cm] : 0u;
        const uint32_t s = cm < ncells ? start[cm] : 0u;
        const uint32_t cnt0 = __shfl_sync(FULL, cnt, 0), cnt1 = __shfl_sync(FULL, cnt, 16);
        if (max(cnt0, cnt1) <= 16u) {
            const bool mine = (uint32_t)hl < cnt;
            const unsigned long long kq = mine ? tmp_key[s + hl] : ~0ull;  // absent: ranks last
            const int iq = mine ? tmp_idx[s + hl] : 0x7fffffff;
            __syncwarp();
            be[lane] = make_ulonglong2(kq, (unsigned long long)(unsigned)iq);
            __syncwarp();
            const uint32_t rank = rank_in(be + half * 16, max(cnt0, cnt1), kq, iq);
            if (mine)
                put_entry(x, y, w, g, s + rank, iq, kq, xs, ys, zs, ws, pos64, perm, wm);
            continue;
        }
        for (int h = 0; h < 2; ++h) {  // whole warp, one cell after the other
            const uint32_t cn = h ? cnt1 : cnt0;
            const uint32_t sc = __shfl_sync(FULL, s, h * 16);
            if (cn == 0)
                continue;
            const bool buffered = cn <= (uint32_t)SORT_BUF;
            if (buffered) {
                __syncwarp();
                for (uint32_t e = lane; e < cn; e += 32)
                    be[e] = make_ulonglong2(tmp_key[sc + e], (unsigned long long)(unsigned)tmp_idx[sc + e]);
                __syncwarp();
            }
            for (uint32_t e0 = 0; e0 < cn; e0 += 32) {
                const uint32_t e = e0 + lane;
                const bool mine = e < cn;
                unsigned long long kq = ~0ull;
                int iq = 0x7fffffff;
                if (mine) {
                    if (buffered) {
                        kq = be[e].x;
                        iq = (int)be[e].y;
                    } else {
                        kq = tmp_key[sc + e];
                        iq = tmp_idx[sc + e];
                    }
                }
                uint32_t rank = 0;
                if (buffered) {
                    rank = rank_in(be, cn, kq, iq);
                } else {
                    for (uint32_t m = 0; m < cn; ++m) {
                        const unsigned long long km = tmp_key[sc + m];
                        const int im = tmp_idx[sc + m];
                        rank += (km < kq) || (km == kq && im < iq);
                    }
                }
                if (mine)
                    put_entry(x, y, w, g, sc + rank, iq, kq, xs, ys, zs, ws, pos64, perm, wm);
            }
        }
    }
    if (wmax) {  // one atomic per block
        __shared__ unsigned red[SORT_THREADS / 32];
        wm = __reduce_max_sync(FULL, wm);
        if (lane == 0)
            red[wid] = wm;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned m = 0;
            for (int q = 0; q < SORT_THREADS / 32; ++q)
                m = max(m, red[q]);
            atomicMax(wmax, m);
        }
    }
}

// Padding entries at the end of each column: NaN (never counted), perm -1.
__global__ void k_padfill(const uint32_t *__restrict__ start, const uint32_t *__restrict__ pad,
                          int ncols, int nz, float *__restrict__ xs, float *__restrict__ ys,
                          float *__restrict__ zs, float *__restrict__ ws,
                          double4_32a *__restrict__ pos64, int *__restrict__ perm)
{
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncols)
        return;
    const uint32_t e = start[(long long)(col + 1) * nz];
    const float fn = __int_as_float(0x7fc00000);
    const double dn = __longlong_as_double(0x7ff8000000000000ll);
    for (uint32_t q = e - pad[col]; q < e; ++q) {
        xs[q] = ys[q] = zs[q] = fn;
        if (ws)
            ws[q] = 0.0f;
        pos64[q] = make_double4_32a(dn, dn, dn, dn);
        perm[q] = -1;
    }
}

// One block per column: (xmin, xmax, ymin, ymax) of its points, with min / max
// taken on order-preserving integer keys (padding entries, NaN, are skipped).
__global__ void __launch_bounds__(256) k_colbox(const double4_32a *__restrict__ pos64,
                                                const uint32_t *__restrict__ start, int ncols,
                                                int nz, double4_32a *__restrict__ colbox)
{
    __shared__ unsigned long long red[4][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int col = blockIdx.x; col < ncols; col += gridDim.x) {
        const uint32_t s = start[(long long)col * nz], e = start[(long long)(col + 1) * nz];
        unsigned long long x0 = ~0ull, x1 = 0ull, y0 = ~0ull, y1 = 0ull;
        for (uint32_t r = s + threadIdx.x; r < e; r += blockDim.x) {
            const long long bx = __double_as_longlong(pos64[r].x);
            const long long by = __double_as_longlong(pos64[r].y);
            if ((bx & 0x7ff0000000000000ll) == 0x7ff0000000000000ll)
                continue;  // padding
            const unsigned long long kx = order_key(bx), ky = order_key(by);
            x0 = min(x0, kx);
            x1 = max(x1, kx);
            y0 = min(y0, ky);
            y1 = max(y1, ky);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x0 = min(x0, __shfl_xor_sync(FULL, x0, o));
            x1 = max(x1, __shfl_xor_sync(FULL, x1, o));
            y0 = min(y0, __shfl_xor_sync(FULL, y0, o));
            y1 = max(y1, __shfl_xor_sync(FULL, y1, o));
        }
        if (lane == 0) {
            red[0][wid] = x0;
            red[1][wid] = x1;
            red[2][wid] = y0;
            red[3][wid] = y1;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
                x0 = min(x0, red[0][q]);
                x1 = max(x1, red[1][q]);
                y0 = min(y0, red[2][q]);
                y1 = max(y1, red[3][q]);
            }
            // empty column: keys keep their start values; mark the box empty
            colbox[col] = x1 == 0ull ? make_double4_32a(DBL_MAX, -DBL_MAX, DBL_MAX, -DBL_MAX)
                                     : make_double4_32a(key_value(x0), key_value(x1),
                                                        key_value(y0), key_value(y1));
        }
        __syncthreads();
    }
}

// Order-preserving map of a double onto uint64 (for atomic min / max).
__device__ __forceinline__ unsigned long long dkey(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

template <class T>
__global__ void k_bbox(const T *__restrict__ x, const T *__restrict__ y, const T *__restrict__ z,
                       long long n, unsigned long long *__restrict__ out /* 6: min xyz, max xyz */,
                       unsigned *__restrict__ err)
{
    double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    bool bad = false;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const double v[3] = {(double)x[p], (double)y[p], (double)z[p]};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!isfinite(v[a])) {
                bad = true;
                continue;
            }
            lo[a] = fmin(lo[a], v[a]);
            hi[a] = fmax(hi[a], v[a]);
        }
    }
    if (bad)
        atomicOr(err, ERR_COORD);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fmin(lo[a], __shfl_xor_sync(FULL, lo[a], o));
            hi[a] = fmax(hi[a], __shfl_xor_sync(FULL, hi[a], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(&out[a], dkey(lo[a]));
            atomicMax(&out[3 + a], dkey(hi[a]));
        }
    }
}

inline int grid_blocks(long long n, int threads, int sms)
{
    long long b = (n + threads - 1) / threads;
    long long cap = (long long)sms * 16;
    if (b > cap)
        b = cap;
    return (int)(b < 1 ? 1 : b);
}

// Rounding residuals of the float32 frame coordinates, from the sorted binary64
// copies: r = fl32((X - O) - x~) with (X - O) evaluated as the frame conversion
// does (binary64; X itself in a periodic box, whose origin is 0).  The float32
// mean separation uses them to restore the coordinates' lost bits.  Padding
// entries get 0.
__global__ void k_residual(const double4_32a *__restrict__ pos64, const float *__restrict__ xs,
                           const float *__restrict__ ys, const float *__restrict__ zs,
                           const uint32_t *__restrict__ cell_start, Geom g, float *__restrict__ xl,
                           float *__restrict__ yl, float *__restrict__ zl)
{
    const long long n = cell_start[g.ncells];  // padded length of the gridded catalogue
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long d = (long long)blockIdx.x * blockDim.x + threadIdx.x; d < n; d += stride) {
        const double4_32a p = pos64[d];
        if (isnan(p.x)) {
            xl[d] = yl[d] = zl[d] = 0.0f;
            continue;
        }
        const double X = g.periodic ? p.x : __dsub_rn(p.x, g.origin[0]);
        const double Y = g.periodic ? p.y : __dsub_rn(p.y, g.origin[1]);
        const double Z = g.periodic ? p.z : __dsub_rn(p.z, g.origin[2]);
        xl[d] = __double2float_rn(__dsub_rn(X, (double)xs[d]));
        yl[d] = __double2float_rn(__dsub_rn(Y, (double)ys[d]));
        zl[d] = __double2float_rn(__dsub_rn(Z, (double)zs[d]));
    }
}

// ============================================================ batched gridding
// The same stages for every catalogue (segment) of a batch, one launch each:
// a stage's blocks are split among the segments by a prefix array, and the
// counting sort's offsets come from one scan over the segments' concatenated
// padded counts (each segment's ncells + 1 entries, the last one 0), from which
// every segment's cell_start is its slice minus the slice's first value.

// Segment of this block: the largest s with pre[s] <= blockIdx.x (segments
// without blocks of this shape are passed over).  Every thread must call it.
__device__ __forceinline__ int block_seg(const unsigned *pre, int nseg)
{
    __shared__ int s_seg;
    if (threadIdx.x == 0) {
        int lo = 0, hi = nseg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pre[mid] <= blockIdx.x)
                lo = mid;
            else
                hi = mid - 1;
        }
        s_seg = lo;
    }
    __syncthreads();
    return s_seg;
}

// Segment holding entry c of the concatenated per-cell arrays.
__device__ __forceinline__ int seg_of_entry(const GridBatch &B, long long c)
{
    int lo = 0, hi = B.nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.seg[mid].c0 <= c)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) kb_assign(const GridBatch B)
{
    __shared__ Geom g;
    const int s = block_seg(B.pre[GB_POINTS], B.nseg);
    const GridSeg &S = B.seg[s];
    static_assert(sizeof(Geom) % 4 == 0, "geometry copied as words");
    for (int q = threadIdx.x; q < (int)(sizeof(Geom) / 4); q += blockDim.x)
        reinterpret_cast<int *>(&g)[q] = reinterpret_cast<const int *>(B.geom + S.job)[q];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long p = (long long)(blockIdx.x - B.pre[GB_POINTS][s]) * blockDim.x + threadIdx.x;
    const bool live = p < S.n;
    uint32_t cell = 0xffffffffu;
    if (live) {
        float fx, fy, fz;
        bool ok;
        if (S.f32)
            ok = coord(static_cast<const float *>(S.x)[p], 0, g, fx) &
                 coord(static_cast<const float *>(S.y)[p], 1, g, fy) &
                 coord(static_cast<const float *>(S.z)[p], 2, g, fz);
        else
            ok = coord(static_cast<const double *>(S.x)[p], 0, g, fx) &
                 coord(static_cast<const double *>(S.y)[p], 1, g, fy) &
                 coord(static_cast<const double *>(S.z)[p], 2, g, fz);
        if (!ok) {
            atomicOr(S.err, ERR_COORD);
            fx = fy = fz = 0.0f;
        }
        const int cx = cell_index_f(fx, g.inv_wf[0], g.ncx);
        const int cy = cell_index_f(fy, g.inv_wf[1], g.ncy);
        const int cz = cell_index_f(fz, g.inv_wf[2], g.nz);
        cell = (uint32_t)(((long long)(cx * g.ncy + cy)) * g.nz + cz);
    }
    // one segment per block: equal cells are equal entries
    const unsigned same = __match_any_sync(FULL, cell);
    const int leader = __ffs(same) - 1;
    uint32_t b0 = 0;
    if (live && lane == leader)
        b0 = atomicAdd(&B.counts[S.c0 + cell], (uint32_t)__popc(same));
    b0 = __shfl_sync(FULL, b0, leader);
    if (live) {
        S.cell_of[p] = cell;
        S.slot[p] = b0 + (uint32_t)__popc(same & ((1u << lane) - 1u));
    }
}

// One warp per column (as k_colpad), into the concatenated padded counts; the
// last column also zeroes the segment's extra entry.
__global__ void __launch_bounds__(256) kb_colpad(const GridBatch B)
{
    const int s = block_seg(B.pre[GB_COLWARPS], B.nseg);
    const GridSeg &S = B.seg[s];
    const Geom &g = B.geom[S.job];
    const int lane = threadIdx.x & 31, ncols = g.ncols, nz = g.nz;
    const int col = (int)(blockIdx.x - B.pre[GB_COLWARPS][s]) * 8 + (int)(threadIdx.x >> 5);
    if (col >= ncols)
        return;
    const uint32_t *count = B.counts + S.c0;
    uint32_t *padded = B.scan + S.c0;
    const long long c0 = (long long)col * nz;
    uint32_t tot = 0;
    for (int z = lane; z < nz; z += 32) {
        const uint32_t v = count[c0 + z];
        padded[c0 + z] = v;
        tot += v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        tot += __shfl_xor_sync(FULL, tot, o);
    const uint32_t pd = (4u - (tot & 3u)) & 3u;
    __syncwarp();
    if (lane == 0) {
        S.pad[col] = pd;
        padded[c0 + nz - 1] += pd;
        if (col == ncols - 1)
            padded[g.ncells] = 0u;
    }
}

// cell_start of every segment: its slice of the scan minus the slice's first value.
__global__ void __launch_bounds__(256) kb_cellstart(const GridBatch B)
{
    const int s = block_seg(B.pre[GB_CELLS], B.nseg);
    const GridSeg &S = B.seg[s];
    const long long k = (long long)(blockIdx.x - B.pre[GB_CELLS][s]) * blockDim.x + threadIdx.x;
    if (k <= B.geom[S.job].ncells)
        S.out.cell_start[k] = B.scan[S.c0 + k] - B.scan[S.c0];
}

__global__ void __launch_bounds__(256) kb_scatter(const GridBatch B)
{
    const int s = block_seg(B.pre[GB_POINTS], B.nseg);
    const GridSeg &S = B.seg[s];
    const long long p = (long long)(blockIdx.x - B.pre[GB_POINTS][s]) * blockDim.x + threadIdx.x;
    if (p >= S.n)
        return;
    const uint32_t q = S.out.cell_start[S.cell_of[p]] + S.slot[p];
    const double zv = S.f32 ? (double)static_cast<const float *>(S.z)[p] : static_cast<const double *>(S.z)[p];
    S.tmp_idx[q] = (int)p;
    S.tmp_key[q] = order_key(__double_as_longlong(zv));
}

__device__ __forceinline__ void put_seg(const GridBatch &B, const GridSeg &S, uint32_t d, int iq,
                                        unsigned long long kq, unsigned &wm)
{
    const Geom &g = B.geom[S.job];
    if (S.f32)
        put_entry(static_cast<const float *>(S.x), static_cast<const float *>(S.y), nullptr, g, d, iq,
                  kq, S.out.xs, S.out.ys, S.out.zs, nullptr, S.out.pos64, S.out.perm, wm);
    else
        put_entry(static_cast<const double *>(S.x), static_cast<const double *>(S.y), nullptr, g, d,
                  iq, kq, S.out.xs, S.out.ys, S.out.zs, nullptr, S.out.pos64, S.out.perm, wm);
}

// k_sort_cells over the concatenated cells of every segment (the two cells of
// a claim may belong to different segments; a segment's extra entry has no
// points).
__global__ void __launch_bounds__(SORT_THREADS) kb_sort_cells(const GridBatch B)
{
    __shared__ ulonglong2 s_ent[SORT_THREADS / 32][SORT_BUF];
    const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15, wid = threadIdx.x >> 5;
    ulonglong2 *be = s_ent[wid];
    unsigned wm = 0;
    for (;;) {
        unsigned v = 0u;
        if (lane == 0)
            v = atomicAdd(B.counts + B.ctot, 1u);  // the next pair of entries (zeroed with the counts)
        const long long c0 = 2ll * __shfl_sync(FULL, v, 0);
        if (c0 >= B.ctot)
            break;
        const long long cm = c0 + half;  // this half warp's entry
        int sg = 0;
        uint32_t cnt = 0u, s0 = 0u;
        if (cm < B.ctot) {
            sg = seg_of_entry(B, cm);
            cnt = B.counts[cm];
            if (cnt)
                s0 = B.seg[sg].out.cell_start[cm - B.seg[sg].c0];
        }
        const uint32_t cnt0 = __shfl_sync(FULL, cnt, 0), cnt1 = __shfl_sync(FULL, cnt, 16);
        if (max(cnt0, cnt1) <= 16u) {
            const GridSeg &S = B.seg[sg];
            const bool mine = (uint32_t)hl < cnt;
            const unsigned long long kq = mine ? S.tmp_key[s0 + hl] : ~0ull;
            const int iq = mine ? S.tmp_idx[s0 + hl] : 0x7fffffff;
            __syncwarp();
            be[lane] = make_ulonglong2(kq, (unsigned long long)(unsigned)iq);
            __syncwarp();
            const uint32_t rank = rank_in(be + half * 16, max(cnt0, cnt1), kq, iq);
            if (mine)
                put_seg(B, S, s0 + rank, iq, kq, wm);
            continue;
        }
        for (int h = 0; h < 2; ++h) {  // whole warp, one cell after the other
            const uint32_t cn = h ? cnt1 : cnt0;
            const uint32_t sc = __shfl_sync(FULL, s0, h * 16);
            const int sh = __shfl_sync(FULL, sg, h * 16);
            if (cn == 0)
                continue;
            const GridSeg &S = B.seg[sh];
            const bool buffered = cn <= (uint32_t)SORT_BUF;
            if (buffered) {
                __syncwarp();
                for (uint32_t e = lane; e < cn; e += 32)
                    be[e] = make_ulonglong2(S.tmp_key[sc + e], (unsigned long long)(unsigned)S.tmp_idx[sc + e]);
                __syncwarp();
            }
            for (uint32_t e0 = 0; e0 < cn; e0 += 32) {
                const uint32_t e = e0 + lane;
                const bool mine = e < cn;
                unsigned long long kq = ~0ull;
                int iq = 0x7fffffff;
                if (mine) {
                    if (buffered) {
                        kq = be[e].x;
                        iq = (int)be[e].y;
                    } else {
                        kq = S.tmp_key[sc + e];
                        iq = S.tmp_idx[sc + e];
                    }
                }
                uint32_t rank = 0;
                if (buffered) {
                    rank = rank_in(be, cn, kq, iq);
                } else {
                    for (uint32_t m = 0; m < cn; ++m) {
                        const unsigned long long km = S.tmp_key[sc + m];
                        const int im = S.tmp_idx[sc + m];
                        rank += (km < kq) || (km == kq && im < iq);
                    }
                }
                if (mine)
                    put_seg(B, S, sc + rank, iq, kq, wm);
            }
        }
    }
}

__global__ void __launch_bounds__(256) kb_padfill(const GridBatch B)
{
    const int s = block_seg(B.pre[GB_COLS], B.nseg);
    const GridSeg &S = B.seg[s];
    const Geom &g = B.geom[S.job];
    const int col = (int)(blockIdx.x - B.pre[GB_COLS][s]) * 256 + (int)threadIdx.x;
    if (col >= g.ncols)
        return;
    const uint32_t e = S.out.cell_start[(long long)(col + 1) * g.nz];
    const float fn = __int_as_float(0x7fc00000);
    const double dn = __longlong_as_double(0x7ff8000000000000ll);
    for (uint32_t q = e - S.pad[col]; q < e; ++q) {
        S.out.xs[q] = S.out.ys[q] = S.out.zs[q] = fn;
        S.out.pos64[q] = make_double4_32a(dn, dn, dn, dn);
        S.out.perm[q] = -1;
    }
}

// One block per column (as k_colbox).
__global__ void __launch_bounds__(256) kb_colbox(const GridBatch B)
{
    __shared__ unsigned long long red[4][8];
    const int s = block_seg(B.pre[GB_COLBLK], B.nseg);
    const GridSeg &S = B.seg[s];
    const int nz = B.geom[S.job].nz;
    const int col = (int)(blockIdx.x - B.pre[GB_COLBLK][s]);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t st = S.out.cell_start[(long long)col * nz], en = S.out.cell_start[(long long)(col + 1) * nz];
    unsigned long long x0 = ~0ull, x1 = 0ull, y0 = ~0ull, y1 = 0ull;
    for (uint32_t r = st + threadIdx.x; r < en; r += blockDim.x) {
        const long long bx = __double_as_longlong(S.out.pos64[r].x);
        const long long by = __double_as_longlong(S.out.pos64[r].y);
        if ((bx & 0x7ff0000000000000ll) == 0x7ff0000000000000ll)
            continue;  // padding
        const unsigned long long kx = order_key(bx), ky = order_key(by);
        x0 = min(x0, kx);
        x1 = max(x1, kx);
        y0 = min(y0, ky);
        y1 = max(y1, ky);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x0 = min(x0, __shfl_xor_sync(FULL, x0, o));
        x1 = max(x1, __shfl_xor_sync(FULL, x1, o));
        y0 = min(y0, __shfl_xor_sync(FULL, y0, o));
        y1 = max(y1, __shfl_xor_sync(FULL, y1, o));
    }
    if (lane == 0) {
        red[0][wid] = x0;
        red[1][wid] = x1;
        red[2][wid] = y0;
        red[3][wid] = y1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
            x0 = min(x0, red[0][q]);
            x1 = max(x1, red[1][q]);
            y0 = min(y0, red[2][q]);
            y1 = max(y1, red[3][q]);
        }
        S.out.colbox[col] = x1 == 0ull ? make_double4_32a(DBL_MAX, -DBL_MAX, DBL_MAX, -DBL_MAX)
                                       : make_double4_32a(key_value(x0), key_value(x1),
                                                          key_value(y0), key_value(y1));
    }
}

template <class T>
cudaError_t build_grid_t(const void *x, const void *y, const void *z, const double *w, long long n,
                         const Geom &g, const GridTemps &t, Gridded &out, int sms, unsigned *err,
                         cudaStream_t st)
{
    cudaError_t e;
    const long long nc = g.ncells;
    if ((e = cudaMemsetAsync(t.counts, 0, sizeof(uint32_t) * (nc + 1), st)))  // + the sort's claim counter
        return e;
    const int TB = 256;
    if (n > 0) {
        k_assign<T><<<grid_blocks(n, TB, sms), TB, 0, st>>>((const T *)x, (const T *)y,
                                                            (const T *)z, n, g, t.cell_of, t.slot,
                                                            t.counts, err);
    }
    const int cb = (g.ncols * 32 + 255) / 256;
    k_colpad<<<cb, 256, 0, st>>>(t.counts, g.ncols, g.nz, t.pad, out.cell_start);
    const int nb = (int)((nc + SCAN_ITEMS - 1) / SCAN_ITEMS);
    k_scan_blocks<<<nb, SCAN_THREADS, 0, st>>>(out.cell_start, out.cell_start, nc, t.bsum);
    k_scan_sums<<<1, SCAN_THREADS, 0, st>>>(t.bsum, (long long)nb, out.cell_start + nc);
    k_scan_add<<<(int)((nc + 255) / 256), 256, 0, st>>>(out.cell_start, nc, t.bsum);
    if (n > 0) {
        k_scatter<T><<<grid_blocks(n, TB, sms), TB, 0, st>>>((const T *)z, n, t.cell_of, t.slot,
                                                             out.cell_start, t.tmp_idx, t.tmp_key);
        const long long cwarps = std::min<long long>((nc + 1) / 2, (long long)sms * 64);
        k_sort_cells<T><<<(int)((cwarps * 32 + SORT_THREADS - 1) / SORT_THREADS), SORT_THREADS, 0, st>>>(
            (const T *)x, (const T *)y, w, nc, g, t.counts, out.cell_start, t.tmp_idx, t.tmp_key,
            out.xs, out.ys, out.zs, out.ws, out.ws ? out.wmax : nullptr, out.pos64, out.perm,
            t.counts + nc);
    }
    k_padfill<<<(g.ncols + 255) / 256, 256, 0, st>>>(out.cell_start, t.pad, g.ncols, g.nz, out.xs,
                                                      out.ys, out.zs, out.ws, out.pos64, out.perm);
    k_colbox<<<std::min(g.ncols, sms * 8), 256, 0, st>>>(out.pos64, out.cell_start, g.ncols, g.nz,
                                                          out.colbox);
    if (out.xl) {
        const long long np = n + 3ll * g.ncols;  // padded length (an upper bound)
        k_residual<<<grid_blocks(np, TB, sms), TB, 0, st>>>(out.pos64, out.xs, out.ys, out.zs,
                                                            out.cell_start, g, out.xl, out.yl,
                                                            out.zl);
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t bbox_t(const void *x, const void *y, const void *z, long long n,
                   unsigned long long *out6, int sms, unsigned *err, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    k_bbox<T><<<grid_blocks(n, 256, sms), 256, 0, st>>>((const T *)x, (const T *)y, (const T *)z, n,
                                                         out6, err);
    return cudaGetLastError();
}

}  // namespace

cudaError_t build_grid(cf_dtype dt, const void *x, const void *y, const void *z, const double *w,
                       long long n, const Geom &g, const GridTemps &t, Gridded &out, int sms,
                       unsigned *err, cudaStream_t st)
{
    out.n = n;
    return dt == CF_FLOAT32 ? build_grid_t<float>(x, y, z, w, n, g, t, out, sms, err, st)
                            : build_grid_t<double>(x, y, z, w, n, g, t, out, sms, err, st);
}

cudaError_t launch_bbox(cf_dtype dt, const void *x, const void *y, const void *z, long long n,
                        unsigned long long *out6, int sms, unsigned *err, cudaStream_t st)
{
    return dt == CF_FLOAT32 ? bbox_t<float>(x, y, z, n, out6, sms, err, st)
                            : bbox_t<double>(x, y, z, n, out6, sms, err, st);
}

long long scan_block_sums(long long n)
{
    return (n + SCAN_ITEMS - 1) / SCAN_ITEMS + 1;  // + the grand total
}

unsigned grid_batch_blocks(int k, long long n, const Geom &g)
{
    switch (k) {
    case GB_POINTS:
        return (unsigned)((n + 255) / 256);
    case GB_COLWARPS:
        return (unsigned)((g.ncols + 7) / 8);
    case GB_COLS:
        return (unsigned)((g.ncols + 255) / 256);
    case GB_COLBLK:
        return (unsigned)g.ncols;
    default:
        return (unsigned)((g.ncells + 1 + 255) / 256);
    }
}

cudaError_t build_grid_batch(const GridBatch &B, int sms, cudaStream_t st)
{
    cudaError_t e;
    if (B.nseg < 1 || B.ctot < 1)
        return cudaSuccess;
    if ((e = cudaMemsetAsync(B.counts, 0, sizeof(uint32_t) * (B.ctot + 1), st)))  // + the sort's claim counter
        return e;
    if (B.blocks[GB_POINTS])
        kb_assign<<<B.blocks[GB_POINTS], 256, 0, st>>>(B);
    kb_colpad<<<B.blocks[GB_COLWARPS], 256, 0, st>>>(B);
    const long long nb = (B.ctot + SCAN_ITEMS - 1) / SCAN_ITEMS;
    k_scan_blocks<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(B.scan, B.scan, B.ctot, B.bsum);
    k_scan_sums<<<1, SCAN_THREADS, 0, st>>>(B.bsum, nb, B.bsum + nb);
    k_scan_add<<<(unsigned)((B.ctot + 255) / 256), 256, 0, st>>>(B.scan, B.ctot, B.bsum);
    kb_cellstart<<<B.blocks[GB_CELLS], 256, 0, st>>>(B);
    if (B.blocks[GB_POINTS]) {
        kb_scatter<<<B.blocks[GB_POINTS], 256, 0, st>>>(B);
        const long long cwarps = std::min<long long>((B.ctot + 1) / 2, (long long)sms * 64);
        kb_sort_cells<<<(unsigned)((cwarps * 32 + SORT_THREADS - 1) / SORT_THREADS), SORT_THREADS, 0, st>>>(B);
    }
    kb_padfill<<<B.blocks[GB_COLS], 256, 0, st>>>(B);
    kb_colbox<<<B.blocks[GB_COLBLK], 256, 0, st>>>(B);
    return cudaGetLastError();
}

double decode_dkey(unsigned long long k)
{
    const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    double v;
    memcpy(&v, &b, sizeof(v));
    return v;
}

}  // namespace cf
