// Pair kernels: the hot loop of cell-list pair counting (arXiv:1911.08275,
// Sec. 2.2: late entry / early exit on the z-sorted axis, Code 2; distance
// masks on squared separations, Code 3; histogram update by comparing against
// squared edges, Code 4), re-designed for GB300.
//
// Work unit = one (primary column a, secondary column b, periodic image) pair
// ("column pair"); columns are z-sorted (grid.cu).  A persistent CTA pulls
// column pairs from a global counter, drops those whose bounding boxes are at
// least Rmax apart in (x, y) (Sec. 2.2), stages column b into shared memory
// with 1-D TMA bulk copies (cp.async.bulk + mbarrier) in tiles, and its 8 warps
// sweep column a in chunks of I z-consecutive points.  For each chunk and
// periodic z image a warp finds, by a lane-parallel search of the staged z
// values, the window of b points whose z can be within the reach of the chunk
// (the paper's late entry and early exit, applied per chunk rather than per
// particle), then evaluates I x (32/I) pairs per step.
//
// Binning (xi, float32 mode): the squared distance is evaluated in float32;
// its bit pattern indexes a lookup table built on the host from float32
// thresholds lo_k < e_k^2 < hi_k that bracket every squared edge by a proven
// error bound.  A table cell wholly between hi_k and lo_{k+1} gives the bin
// directly; a cell that touches a band falls back to threshold compares, and a
// distance inside a band is re-evaluated with the canonical binary64 formula
// from the binary64 copies of the two points.  Counts are thus bit-identical to
// the binary64 definition.  Each lane owns one column of its warp's histogram
// in shared memory (no atomics, no bank conflicts); columns are reduced and
// added to the global histogram once per CTA.
//
// The binary64 path (CF_MODE_FP64) runs the same loop on binary64 copies with
// the canonical formula and exact squared-edge compares.
#include <cuda_runtime.h>

#include <type_traits>

#include "cf_internal.cuh"
#include "pairs.cuh"

namespace cf {

int pair_hist_words(int kind, int nbins, int npibins)
{
    if (kind == 0)
        return WARPS * nbins * 32;
    return WARPS * nbins * npibins;
}

namespace {

constexpr unsigned WAIT_LIMIT = 1u << 22;

__device__ __forceinline__ int floor_div(int a, int n)
{
    return a >= 0 ? a / n : -((-a + n - 1) / n);
}

// First index p in [0, n) with t[p].z >= v (upper = false) or t[p].z > v
// (upper = true); n if none.  t[0..n) must be sorted by z.  All lanes call it
// with the same arguments; each round probes 32 positions.
template <class P4, class V>
__device__ __forceinline__ int warp_bound(const P4 *t, int n, V v, bool upper, int lane)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int s = (hi - lo + 31) >> 5;
        const int p = lo + lane * s;
        bool q = false;
        if (p < hi) {
            const V z = t[p].z;
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

__device__ __forceinline__ double canon_r2(const double4_32a &p, const double4_32a &q, double Sx, double Sy,
                                           double Sz)
{
    const double dx = canon_comp(p.x, q.x, Sx);
    const double dy = canon_comp(p.y, q.y, Sy);
    const double dz = canon_comp(p.z, q.z, Sz);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Rare path of the float32 binning: the table cell touches an error band.
// Returns 1 if the pair was re-evaluated in binary64.
__device__ __noinline__ int bin_slow(uint32_t e, float d2, const float *thr, int nthr, int nb,
                                     const double *E2, uint32_t *hl, const double4_32a *pa,
                                     const double4_32a *pb, int i, int j, double Sx, double Sy,
                                     double Sz)
{
    int c = -1;
    if (e != LUT_AMBIG) {
        c = (int)(e & 0x3fffu);
        while (c < nthr && thr[c] <= d2)
            ++c;
    }
    if (c >= 0 && !(c & 1)) {
        if (c >= 2 && c <= 2 * nb)
            hl[((c - 2) >> 1) * 32] += 1u;
        return 0;
    }
    const double r2 = canon_r2(pa[i], pb[j], Sx, Sy, Sz);
    const int k = bin_f64(r2, E2, nb);
    if (k >= 0)
        hl[k * 32] += 1u;
    return 1;
}

// Debug: does the float32 decision for d2 agree with binary64?  (1 = violation)
__device__ __noinline__ int verify_pair(float d2, const float *thr, int nthr, int nb,
                                        const double *E2, const double4_32a *pa, const double4_32a *pb,
                                        int i, int j, double Sx, double Sy, double Sz)
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

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
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
        const unsigned long long v = warp_sum_u64(hw[b * 32 + lane]);
        hw[b * 32 + lane] = 0u;
        if (lane == 0 && v)
            atomicAdd(&ghist[b], v);
    }
}

template <bool F64, int I, bool EVALS, bool VERIFY>
__global__ void __launch_bounds__(THREADS) k_xi(const __grid_constant__ PairParams P)
{
    using P4 = typename std::conditional<F64, double4_32a, float4>::type;
    using V = typename std::conditional<F64, double, float>::type;
    constexpr int J = 32 / I;
    extern __shared__ __align__(128) unsigned char smem[];

    const int nb = P.nbins;
    const SmemLayout L = smem_layout(P.tile_max, (int)sizeof(P4), F64 ? 0 : P.lut_n,
                                     F64 ? 0 : P.nthr, nb, 0, 0, 0, WARPS * nb * 32);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    volatile int *s_item = reinterpret_cast<volatile int *>(smem + 8);
    P4 *tile = reinterpret_cast<P4 *>(smem + L.tile);
    uint16_t *lut = reinterpret_cast<uint16_t *>(smem + L.lut);
    float *thr = reinterpret_cast<float *>(smem + L.thr);
    double *E2 = reinterpret_cast<double *>(smem + L.e2);
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem + L.hist);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (!F64) {
        for (int q = tid; q < P.lut_n; q += THREADS)
            lut[q] = P.lut[q];
        for (int q = tid; q < P.nthr; q += THREADS)
            thr[q] = P.thr[q];
    }
    for (int q = tid; q <= nb; q += THREADS)
        E2[q] = P.E2[q];
    for (int q = tid; q < WARPS * nb * 32; q += THREADS)
        hist[q] = 0u;
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();

    uint32_t *hw = hist + warp * nb * 32;
    uint32_t *hl = hw + lane;
    const int ii = lane % I, jj = lane / I;
    unsigned phase = 0;
    unsigned long long n_eval = 0, n_rck = 0, n_viol = 0;
    unsigned pending = 0;
    bool aborted = false;
    const double4_32a *pa64 = P.A.pos64, *pb64 = P.B.pos64;

    for (;;) {
        if (tid == 0)
            *s_item = (int)atomicAdd(P.item_counter, 1u);
        __syncthreads();
        const int item = *s_item;
        __syncthreads();
        if (item >= P.n_items)
            break;
        const int a = item / P.nstencil, s = item - a * P.nstencil;
        const int2 o = P.stencil[s];
        const int ax = a / P.g.ncy, ay = a - ax * P.g.ncy;
        int bx = ax + o.x, by = ay + o.y;
        double Sx = 0.0, Sy = 0.0;
        if (P.g.periodic) {
            const int qx = floor_div(bx, P.g.ncx), qy = floor_div(by, P.g.ncy);
            bx -= qx * P.g.ncx;
            by -= qy * P.g.ncy;
            Sx = qx * P.g.box[0];
            Sy = qy * P.g.box[1];
        } else if (bx < 0 || bx >= P.g.ncx || by < 0 || by >= P.g.ncy) {
            continue;
        }
        const int b = bx * P.g.ncy + by;
        const long long nz = P.g.nz;
        const int a0 = (int)P.A.cell_start[a * nz], a1 = (int)P.A.cell_start[(a + 1) * nz];
        const int b0 = (int)P.B.cell_start[b * nz], b1 = (int)P.B.cell_start[(b + 1) * nz];
        if (a0 >= a1 || b0 >= b1)
            continue;
        // Sec. 2.2: minimum possible (x, y) separation of the two columns' boxes.
        const double4_32a ba = P.A.colbox[a], bb = P.B.colbox[b];
        const double gx = fmax(0.0, fmax(__dsub_rn(__dadd_rn(bb.x, Sx), ba.y),
                                         __dsub_rn(ba.x, __dadd_rn(bb.y, Sx))));
        const double gy = fmax(0.0, fmax(__dsub_rn(__dadd_rn(bb.z, Sy), ba.w),
                                         __dsub_rn(ba.z, __dadd_rn(bb.w, Sy))));
        const double g2 = __dadd_rn(__dmul_rn(gx, gx), __dmul_rn(gy, gy));
        if (!(P.flags & CF_FLAG_NO_PRUNE) && g2 >= P.prune_r2)
            continue;
        // z reach of this column pair: dz_max,all of Sec. 2.2 (xi), pimax (rp-pi).
        double dzmax = P.rz;
        if (P.kind == 0)
            dzmax = sqrt(fmax(0.0, __dsub_rn(P.rxy2, __dmul_rn(g2, 1.0 - 1e-12))));
        dzmax = __dmul_rn(dzmax, 1.0 + 1e-9);
        V dzw;
        if (F64)
            dzw = (V)__dadd_rn(dzmax, 1e-9 * (P.rz + P.g.box[2] + 1.0));
        else
            dzw = (V)__fadd_ru(__double2float_ru(dzmax), P.zslack);
        const bool self = P.autocorr && o.x == 0 && o.y == 0;
        const int kmin = P.g.periodic ? (self ? 0 : -1) : 0;
        const int kmax = P.g.periodic ? 1 : 0;
        if (tid == 0)
            atomicAdd(&P.diag[0], 1ull);
        const float Sxf = __double2float_rn(Sx), Syf = __double2float_rn(Sy);
        const int na = a1 - a0;
        const int nchunks = (na + I - 1) / I;

        for (int t0 = b0; t0 < b1 && !aborted; t0 += P.tile_max) {
            const int nt = min(P.tile_max, b1 - t0);
            __syncthreads();  // previous tile fully consumed
            if (tid == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar, (unsigned)(nt * sizeof(P4)));
                const void *src = F64 ? (const void *)(P.B.pos64 + t0) : (const void *)(P.B.pos + t0);
                bulk_g2s(tile, src, (unsigned)(nt * sizeof(P4)), bar);
            }
            if (tid < 32) {
                P4 nanp;
                nanp.x = nanp.y = nanp.z = nanp.w = (V)__int_as_float(0x7fc00000);
                tile[nt + tid] = nanp;  // sentinels: never counted
            }
            const bool ok = mbar_wait(bar, phase, WAIT_LIMIT);
            phase ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (tid == 0)
                    atomicOr(P.err, ERR_TIMEOUT);
                aborted = true;
                break;
            }
            const V zt_lo = tile[0].z, zt_hi = tile[nt - 1].z;

            for (int c = warp; c < nchunks; c += WARPS) {
                const int ib = a0 + c * I;
                const int nvi = min(I, a1 - ib);
                const int i = ib + ii;
                const bool vi = ii < nvi;
                P4 pi;
                if (vi) {
                    if (F64)
                        pi = *reinterpret_cast<const P4 *>(&pa64[i]);
                    else
                        pi = *reinterpret_cast<const P4 *>(&P.A.pos[i]);
                } else {
                    pi.x = pi.y = pi.z = pi.w = (V)__int_as_float(0x7fc00000);
                }
                const V zlo = __shfl_sync(FULL, pi.z, 0);
                const V zhi = __shfl_sync(FULL, pi.z, nvi - 1);
                const float xh = F64 ? 0.f : __fsub_rn((float)pi.x, Sxf);
                const float yh = F64 ? 0.f : __fsub_rn((float)pi.y, Syf);
                double4_32a pi64 = make_double4_32a(0, 0, 0, 0);
                if (F64)
                    pi64 = make_double4_32a((double)pi.x, (double)pi.y, (double)pi.z, 0.0);

                for (int k = kmin; k <= kmax; ++k) {
                    const V kz = F64 ? (V)(k * P.g.box[2]) : (V)((float)k * P.boxf[2]);
                    const V wlo = zlo - kz - dzw, whi = zhi - kz + dzw;
                    if (whi < zt_lo || wlo > zt_hi)
                        continue;
                    int jlo = warp_bound(tile, nt, wlo, false, lane);
                    const int jhi = warp_bound(tile, nt, whi, true, lane);
                    const bool tri = self && k == 0;
                    if (tri)
                        jlo = max(jlo, ib + 1 - t0);
                    if (jlo >= jhi)
                        continue;
                    pending += (unsigned)((jhi - jlo + J - 1) / J);
                    const double Sz = k * P.g.box[2];
                    const float zh = F64 ? 0.f : __fsub_rn((float)pi.z, (float)kz);

                    for (int jb = jlo; jb < jhi; jb += J) {
                        const int j = jb + jj;
                        const P4 pj = tile[j];
                        const bool live = !tri || (t0 + j > i);
                        if (EVALS)
                            n_eval += (vi && j < jhi && live) ? 1ull : 0ull;
                        if (F64) {
                            const double4_32a q = make_double4_32a((double)pj.x, (double)pj.y, (double)pj.z, 0.0);
                            double r2 = canon_r2(pi64, q, Sx, Sy, Sz);
                            if (!live)
                                r2 = __longlong_as_double(0x7ff8000000000000ll);
                            const int kb = bin_f64(r2, E2, nb);
                            if (kb >= 0)
                                hl[kb * 32] += 1u;
                        } else {
                            const float dx = __fsub_rn((float)pj.x, xh);
                            const float dy = __fsub_rn((float)pj.y, yh);
                            const float dz = __fsub_rn((float)pj.z, zh);
                            float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
                            if (!live)
                                d2 = __int_as_float(0x7fc00000);
                            const uint32_t u = __float_as_uint(d2) - P.u0;
                            if (u < P.urange) {
                                const uint32_t e = lut[u >> P.lut_shift];
                                if (e < 0x4000u)
                                    hl[e >> 2] += 1u;
                                else
                                    n_rck += bin_slow(e, d2, thr, P.nthr, nb, E2, hl, pa64, pb64,
                                                      i, t0 + j, Sx, Sy, Sz);
                            }
                            if (VERIFY && vi && j < nt && live)
                                n_viol += verify_pair(d2, thr, P.nthr, nb, E2, pa64, pb64, i,
                                                      t0 + j, Sx, Sy, Sz);
                        }
                    }
                }
                if (pending > (1u << 30)) {  // keep every per-lane u32 count far from overflow
                    warp_flush(hw, nb, P.hist, lane);
                    pending = 0;
                }
            }
        }
        if (aborted)
            break;
    }

    __syncthreads();
    for (int bn = tid; bn < nb; bn += THREADS) {
        unsigned long long sum = 0;
        for (int w = 0; w < WARPS; ++w)
            for (int l = 0; l < 32; ++l)
                sum += hist[(w * nb + bn) * 32 + l];
        if (sum)
            atomicAdd(&P.hist[bn], sum);
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

template <bool F64, int I, bool EVALS, bool VERIFY>
cudaError_t launch_xi(const PairParams &P, PairLaunch &L, int sms, cudaStream_t st)
{
    auto kern = k_xi<F64, I, EVALS, VERIFY>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem);
    if (e)
        return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, THREADS, L.smem);
    if (e)
        return e;
    if (occ < 1)
        return cudaErrorInvalidConfiguration;
    long long blocks = (long long)sms * occ;
    if (blocks > P.n_items)
        blocks = P.n_items > 0 ? P.n_items : 1;
    L.blocks = (int)blocks;
    kern<<<L.blocks, THREADS, L.smem, st>>>(P);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pairs(const PairParams &P, PairLaunch &L, int sms, cudaStream_t st)
{
    if (P.kind != 0)
        return cudaErrorNotSupported;
    if (L.f64) {
        if (L.evals)
            return launch_xi<true, 8, true, false>(P, L, sms, st);
        if (L.chunk == 32)
            return launch_xi<true, 32, false, false>(P, L, sms, st);
        return launch_xi<true, 8, false, false>(P, L, sms, st);
    }
    if (L.verify)
        return launch_xi<false, 8, true, true>(P, L, sms, st);
    if (L.evals) {
        if (L.chunk == 16)
            return launch_xi<false, 16, true, false>(P, L, sms, st);
        if (L.chunk == 32)
            return launch_xi<false, 32, true, false>(P, L, sms, st);
        return launch_xi<false, 8, true, false>(P, L, sms, st);
    }
    if (L.chunk == 16)
        return launch_xi<false, 16, false, false>(P, L, sms, st);
    if (L.chunk == 32)
        return launch_xi<false, 32, false, false>(P, L, sms, st);
    return launch_xi<false, 8, false, false>(P, L, sms, st);
}

}  // namespace cf
