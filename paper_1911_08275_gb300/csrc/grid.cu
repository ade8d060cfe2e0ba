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

#include "cf_internal.cuh"
#include "grid.cuh"

namespace cf {

namespace {

__device__ __forceinline__ int cell_index_1d(double v, double origin, double inv_w, int n)
{
    double t = floor(__dmul_rn(__dsub_rn(v, origin), inv_w));
    t = fmin(fmax(t, 0.0), (double)(n - 1));
    return (int)t;
}

template <class T>
__global__ void k_assign(const T *__restrict__ x, const T *__restrict__ y, const T *__restrict__ z,
                         long long n, Geom g, uint32_t *__restrict__ cell_of,
                         uint32_t *__restrict__ slot, uint32_t *__restrict__ count,
                         unsigned *__restrict__ err)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        double X = (double)x[p], Y = (double)y[p], Z = (double)z[p];
        bool ok = isfinite(X) && isfinite(Y) && isfinite(Z);
        if (g.periodic)
            ok = ok && X >= 0.0 && X < g.box[0] && Y >= 0.0 && Y < g.box[1] && Z >= 0.0 &&
                 Z < g.box[2];
        if (!ok) {
            atomicOr(err, ERR_COORD);
            X = g.origin[0];
            Y = g.origin[1];
            Z = g.origin[2];
        }
        const int cx = cell_index_1d(X, g.origin[0], g.inv_w[0], g.ncx);
        const int cy = cell_index_1d(Y, g.origin[1], g.inv_w[1], g.ncy);
        const int cz = cell_index_1d(Z, g.origin[2], g.inv_w[2], g.nz);
        const uint32_t cell = (uint32_t)(((long long)(cx * g.ncy + cy)) * g.nz + cz);
        cell_of[p] = cell;
        slot[p] = atomicAdd(&count[cell], 1u);
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

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_sums(uint32_t *bsum, int nb, uint32_t *grand)
{
    __shared__ uint32_t ws[32];
    __shared__ uint32_t tot;
    uint32_t v[SCAN_PER_THREAD];
    uint32_t s = 0;
    const int base = threadIdx.x * SCAN_PER_THREAD;
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        v[k] = (base + k < nb) ? bsum[base + k] : 0u;
        s += v[k];
    }
    uint32_t pre = block_exclusive_scan(s, ws, &tot);
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        if (base + k < nb)
            bsum[base + k] = pre;
        pre += v[k];
    }
    if (threadIdx.x == 0)
        *grand = tot;
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
                          int *__restrict__ tmp_idx, double *__restrict__ tmp_z)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const uint32_t q = start[cell_of[p]] + slot[p];
        tmp_idx[q] = (int)p;
        tmp_z[q] = (double)z[p];
    }
}

// Rank each point inside its cell by (z, original index) among the cell's real
// entries and write the sorted float32 / binary64 copies.  Work per cell is
// quadratic in its occupancy; z-cells are sized for ~16 points on average.
template <class T>
__global__ void k_sort_gather(const T *__restrict__ x, const T *__restrict__ y,
                              const T *__restrict__ z, const double *__restrict__ w, long long n,
                              Geom g, const uint32_t *__restrict__ cell_of,
                              const uint32_t *__restrict__ count, const uint32_t *__restrict__ start,
                              const int *__restrict__ tmp_idx, const double *__restrict__ tmp_z,
                              float *__restrict__ xs, float *__restrict__ ys,
                              float *__restrict__ zs, double4_32a *__restrict__ pos64,
                              int *__restrict__ perm)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const uint32_t c = cell_of[p];
        const uint32_t s = start[c], e = s + count[c];
        const double X = (double)x[p], Y = (double)y[p], Z = (double)z[p];
        const int iq = (int)p;
        uint32_t rank = 0;
        for (uint32_t r = s; r < e; ++r) {
            const double zr = tmp_z[r];
            const int ir = tmp_idx[r];
            rank += (zr < Z) || (zr == Z && ir < iq);
        }
        const uint32_t d = s + rank;
        const double W = w ? w[p] : 0.0;
        pos64[d] = make_double4_32a(X, Y, Z, W);
        xs[d] = __double2float_rn(__dsub_rn(X, g.origin[0]));
        ys[d] = __double2float_rn(__dsub_rn(Y, g.origin[1]));
        zs[d] = __double2float_rn(__dsub_rn(Z, g.origin[2]));
        perm[d] = iq;
    }
}

// Padding entries at the end of each column: NaN (never counted), perm -1.
__global__ void k_padfill(const uint32_t *__restrict__ start, const uint32_t *__restrict__ pad,
                          int ncols, int nz, float *__restrict__ xs, float *__restrict__ ys,
                          float *__restrict__ zs, double4_32a *__restrict__ pos64,
                          int *__restrict__ perm)
{
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncols)
        return;
    const uint32_t e = start[(long long)(col + 1) * nz];
    const float fn = __int_as_float(0x7fc00000);
    const double dn = __longlong_as_double(0x7ff8000000000000ll);
    for (uint32_t q = e - pad[col]; q < e; ++q) {
        xs[q] = ys[q] = zs[q] = fn;
        pos64[q] = make_double4_32a(dn, dn, dn, dn);
        perm[q] = -1;
    }
}

// One warp per column: (xmin, xmax, ymin, ymax) of its points.
__global__ void k_colbox(const double4_32a *__restrict__ pos64, const uint32_t *__restrict__ start,
                         int ncols, int nz, double4_32a *__restrict__ colbox)
{
    const int lane = threadIdx.x & 31;
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (col >= ncols)
        return;
    const uint32_t s = start[(long long)col * nz], e = start[(long long)(col + 1) * nz];
    double x0 = DBL_MAX, x1 = -DBL_MAX, y0 = DBL_MAX, y1 = -DBL_MAX;
    for (uint32_t r = s + lane; r < e; r += 32) {
        const double4_32a p = pos64[r];
        x0 = fmin(x0, p.x);
        x1 = fmax(x1, p.x);
        y0 = fmin(y0, p.y);
        y1 = fmax(y1, p.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x0 = fmin(x0, __shfl_xor_sync(FULL, x0, o));
        x1 = fmax(x1, __shfl_xor_sync(FULL, x1, o));
        y0 = fmin(y0, __shfl_xor_sync(FULL, y0, o));
        y1 = fmax(y1, __shfl_xor_sync(FULL, y1, o));
    }
    if (lane == 0)
        colbox[col] = make_double4_32a(x0, x1, y0, y1);
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

template <class T>
cudaError_t build_grid_t(const void *x, const void *y, const void *z, const double *w, long long n,
                         const Geom &g, const GridTemps &t, Gridded &out, int sms, unsigned *err,
                         cudaStream_t st)
{
    cudaError_t e;
    const long long nc = g.ncells;
    if ((e = cudaMemsetAsync(t.counts, 0, sizeof(uint32_t) * nc, st)))
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
    k_scan_sums<<<1, SCAN_THREADS, 0, st>>>(t.bsum, nb, out.cell_start + nc);
    k_scan_add<<<(int)((nc + 255) / 256), 256, 0, st>>>(out.cell_start, nc, t.bsum);
    if (n > 0) {
        k_scatter<T><<<grid_blocks(n, TB, sms), TB, 0, st>>>((const T *)z, n, t.cell_of, t.slot,
                                                             out.cell_start, t.tmp_idx, t.tmp_z);
        k_sort_gather<T><<<grid_blocks(n, TB, sms), TB, 0, st>>>(
            (const T *)x, (const T *)y, (const T *)z, w, n, g, t.cell_of, t.counts,
            out.cell_start, t.tmp_idx, t.tmp_z, out.xs, out.ys, out.zs, out.pos64, out.perm);
    }
    k_padfill<<<(g.ncols + 255) / 256, 256, 0, st>>>(out.cell_start, t.pad, g.ncols, g.nz, out.xs,
                                                      out.ys, out.zs, out.pos64, out.perm);
    k_colbox<<<cb, 256, 0, st>>>(out.pos64, out.cell_start, g.ncols, g.nz, out.colbox);
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

double decode_dkey(unsigned long long k)
{
    const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    double v;
    memcpy(&v, &b, sizeof(v));
    return v;
}

}  // namespace cf
