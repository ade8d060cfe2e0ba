// C ABI of cfgpu (include/cf.h): argument checks, grid planning, the float32
// error bands, workspace management and the stream-ordered sequence
//   [H2D of host inputs] -> bbox (open boxes) -> grid D1 [, grid D2] ->
//   pair kernel -> D2H of the histogram -> one stream synchronisation.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "cf.h"
#include "cf_internal.cuh"
#include "grid.cuh"
#include "pairs.cuh"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? CF_ENOMEM : CF_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CF_CUDA(call, what)                 \
    do {                                    \
        cudaError_t e_ = (call);            \
        if (e_ != cudaSuccess) {            \
            rc = cuda_fail(e_, what);       \
            goto cleanup;                   \
        }                                   \
    } while (0)

const double U32 = std::ldexp(1.0, -24);
const double U64 = std::ldexp(1.0, -53);

bool is_device_ptr(const void *p)
{
    if (!p)
        return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

float f32_down(double v)
{
    float f = (float)v;
    if ((double)f > v)
        f = std::nextafter(f, -INFINITY);
    return f;
}

float f32_up(double v)
{
    float f = (float)v;
    if ((double)f < v)
        f = std::nextafter(f, INFINITY);
    return f;
}

uint32_t fbits(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
}

float bitsf(uint32_t u)
{
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// Error model of the float32 path:
//   coordinates are fl32(X - O) with |X - O| <= M; the primary is shifted by
//   fl32(S), |S| <= Ls (periodic image), then dx = fl32(x_j - x^_i).
// Per-axis bound on |dx~ - dx_true| for a component of size <= r:
double eps_axis(double r, double M, double Ls)
{
    const double u = U32;
    double E = 2.0 * (u + 2.0 * U64) * M;
    if (Ls > 0)
        E += u * Ls + u * (1.0 + u) * (M + Ls);
    return E * (1.0 + u) + u * (r + E);
}

// Bound on |d2~(float32) - d2(canonical binary64)| for squared separations near S
// (3 components for xi, 2 for rp).  Doubled for safety.
double band_sq(double S, int ncomp, double M, double Ls, double R)
{
    const double u = U32;
    const double s = S * (1.0 + 1e-6);
    const double r = std::sqrt(s);
    const double eps = eps_axis(r, M, Ls);
    const double sq = std::sqrt((double)ncomp);
    const double g = ncomp * u / (1.0 - ncomp * u);
    const double smax = s + 2.0 * eps * sq * r + ncomp * eps * eps;
    double B = g * smax + 2.0 * eps * sq * r + ncomp * eps * eps;
    const double e64 = 2.0 * U64 * (M + Ls + 2.0 * R);
    B += (ncomp + 0.5) * U64 * s + 2.0 * e64 * sq * r + ncomp * e64 * e64;
    return 2.0 * B + 1e-37;
}

// Float32 decision tables for squared separations (ncomp = 3 for xi, 2 for rp).
//   T[0..2*ne): lo_0, hi_0, ..., lo_n, hi_n around the squared edges E2[0..ne):
//     d2~ < lo_k proves d2 < E2_k and d2~ >= hi_k proves d2 >= E2_k.
//   tab[0..lut_n): one byte per cell of float bit patterns; cell q holds the
//     patterns u with (u >> shift) == u0s + q; tab[lut_n - 1] is the entry that
//     every out-of-range distance (below lo_0, at or above hi_n, NaN) uses.
//     Entries: bin k if every value of the cell lies in [hi_k, lo_{k+1});
//     nbins if every value is surely not counted; TAB_FLAGGED otherwise (the
//     cell contains a threshold or lies inside a band).
struct Tables {
    int nthr, lut_n, shift;
    uint32_t u0s;  // first cell's bit pattern >> shift (logarithmic cells)
    int lin;       // 1: cells linear in d2, cell = round(d2 * lscale)
    float lscale;
};

// pi bins: the kernels take t' = fl32(|dz~| * pscale - 1/2), pscale = fl32(npibins / pimax),
// bin m = round(t') and trust it when |t' - m| <= pband.
void pi_band(double pimax, int npibins, double M, double Ls, float &pscale, float &pband)
{
    const double s = (double)npibins / pimax;
    pscale = (float)s;
    // t = |dz| * s: float32 error in t (dz error, the scale's and the fma's
    // roundings, the binary64 edges' own rounding), doubled for safety.
    const double tmax = npibins + 1.0;
    const double eps_z = eps_axis(pimax * (1.0 + 1e-6), M, Ls) + 2.0 * U64 * (M + Ls + 2.0 * pimax);
    const double beta = 2.0 * (eps_z * s * (1.0 + 1e-6) + (2.0 * tmax + 2.0) * U32 +
                               4.0 * tmax * U64) + 1e-30;
    pband = 0.5 - beta > 0.0 ? f32_down(0.5 - beta) : -1.0f;  // -1: every pair re-checked
}

// Thresholds T[0..2 ne) (see above).
void build_thresholds(const double *E2, int ne, int ncomp, double M, double Ls, double R, float *T)
{
    const int nthr = 2 * ne;
    for (int k = 0; k < ne; ++k) {
        if (E2[k] == 0.0) {  // every d2 >= 0 is surely >= 0
            T[2 * k] = 0.0f;
            T[2 * k + 1] = 0.0f;
            continue;
        }
        const double B = band_sq(E2[k], ncomp, M, Ls, R);
        const double lo = E2[k] - B;
        // Near zero the bound is not monotone in d2: never claim "below" there.
        T[2 * k] = (lo <= 0.0 || E2[k] < 1e-6) ? -1.0f : f32_down(lo);
        T[2 * k + 1] = std::nextafter(f32_up(E2[k] + B), INFINITY);
    }
    for (int q = 1; q < nthr; ++q)  // raising a threshold only widens the re-check set
        T[q] = std::max(T[q], T[q - 1]);
}

// Classify cells [vlo[q], vhi[q]] (increasing, closed) against the thresholds;
// returns the pair mass of the flagged cells under the density w(v) = v^(1/2)
// (separations in 3-D) or 1 (rp^2 in 2-D), up to a constant.
template <class Bounds>
double classify_cells(const float *T, int nthr, int nbins, int n, int ncomp, Bounds bounds,
                      uint8_t *tab)
{
    const uint8_t dummy = (uint8_t)nbins, flagged = cf::TAB_FLAGGED;
    auto mass = [&](double a, double b) {
        a = std::max(a, 0.0);
        b = std::max(b, a);
        return ncomp == 3 ? (std::pow(b, 1.5) - std::pow(a, 1.5)) : (b - a);
    };
    double fm = 0.0;
    // Cells are visited in increasing value, so the threshold counts at the cell
    // ends only move forward: one sweep over cells and thresholds.
    int clo = 0, chi = 0;
    for (int q = 0; q < n; ++q) {
        double vlo, vhi;
        bounds(q, vlo, vhi);
        while (clo < nthr && (double)T[clo] <= vlo)
            ++clo;
        chi = std::max(chi, clo);
        while (chi < nthr && (double)T[chi] <= vhi)
            ++chi;
        if (clo == chi && !(clo & 1)) {
            tab[q] = (clo >= 2 && clo <= 2 * nbins) ? (uint8_t)((clo - 2) / 2) : dummy;
        } else {
            tab[q] = flagged;
            fm += mass(vlo, vhi);
        }
    }
    tab[n] = dummy;
    return fm;
}

// Logarithmic cells: cells aligned to multiples of 2^s in the float bit
// pattern, so a kernel finds a value's cell as (bits >> s) - u0s; the last
// cell holds T[nthr - 1].
double log_table(const float *T, int nthr, int nbins, int ncomp, uint8_t *tab, Tables &t)
{
    const uint32_t u0 = T[0] > 0.0f ? fbits(T[0]) : 0u;
    const uint32_t uhi = fbits(T[nthr - 1]);
    int s = 0;
    while (((uhi >> s) - (u0 >> s)) + 1 > (uint32_t)(cf::LUT_MAX - 1))
        ++s;
    const uint32_t u0s = u0 >> s;
    const int n = (int)((uhi >> s) - u0s) + 1;
    const double fm = classify_cells(T, nthr, nbins, n, ncomp, [&](int q, double &lo, double &hi) {
        const uint32_t blo = (u0s + (uint32_t)q) << s;
        lo = bitsf(blo);
        hi = bitsf(blo + (uint32_t)((1ull << s) - 1));
    }, tab);
    t.lut_n = n + 1;
    t.shift = s;
    t.u0s = u0s;
    t.lin = 0;
    t.lscale = 0.0f;
    return fm;
}

// Linear cells: cell q holds the floats v with round(v * lscale) == q (the
// kernel computes it exactly with one fma against 2^23), lscale chosen so that
// the last threshold falls in the last cell; every value above maps past it.
double lin_table(const float *T, int nthr, int nbins, int ncomp, uint8_t *tab, Tables &t)
{
    const int n = cf::LUT_MAX - 1;
    const double top = std::max((double)T[nthr - 1], 1e-30);
    const float ls = f32_down((n - 1.5) / top);
    const double lsd = ls;
    const double out = 1.0 - 1e-12, up = 1.0 + 1e-12;  // closed, slightly widened cell bounds
    const double fm = classify_cells(T, nthr, nbins, n, ncomp, [&](int q, double &lo, double &hi) {
        lo = q == 0 ? 0.0 : (q - 0.5) / lsd * out;
        hi = (q + 0.5) / lsd * up;
    }, tab);
    t.lut_n = n + 1;
    t.shift = 0;
    t.u0s = 0;
    t.lin = 1;
    t.lscale = ls;
    return fm;
}

// Both cell shapes, keeping the one whose flagged cells hold less pair mass.
Tables build_tables(const double *E2, int ne, int ncomp, double M, double Ls, double R, float *T,
                    uint8_t *tab)
{
    Tables tl, tg;
    const int nthr = 2 * ne, nbins = ne - 1;
    build_thresholds(E2, ne, ncomp, M, Ls, R, T);
    tl.nthr = tg.nthr = nthr;
    static thread_local std::vector<uint8_t> other;
    other.resize(cf::LUT_MAX);
    const double fl = lin_table(T, nthr, nbins, ncomp, tab, tl);
    const double fg = log_table(T, nthr, nbins, ncomp, other.data(), tg);
    if (fl <= fg)
        return tl;
    std::memcpy(tab, other.data(), tg.lut_n);
    return tg;
}

// The last tables built on this thread, reused when the inputs repeat (a
// benchmark or an MCMC chain calls with the same bins and box every time).
struct TableCache {
    bool valid = false;
    double key[cf::NB_MAX + 1 + 5];
    int nkey = 0;
    Tables t;
    float T[2 * (cf::NB_MAX + 1)];
    uint8_t tab[cf::LUT_MAX];
};
thread_local TableCache g_tables;

Tables cached_tables(const double *E2, int ne, int ncomp, double M, double Ls, double R, float *T,
                     uint8_t *tab)
{
    TableCache &c = g_tables;
    const int nk = ne + 5;
    bool hit = c.valid && c.nkey == nk;
    const double extra[5] = {(double)ne, (double)ncomp, M, Ls, R};
    for (int k = 0; hit && k < ne; ++k)
        hit = c.key[k] == E2[k];
    for (int k = 0; hit && k < 5; ++k)
        hit = c.key[ne + k] == extra[k];
    if (!hit) {
        c.t = build_tables(E2, ne, ncomp, M, Ls, R, c.T, c.tab);
        for (int k = 0; k < ne; ++k)
            c.key[k] = E2[k];
        for (int k = 0; k < 5; ++k)
            c.key[ne + k] = extra[k];
        c.nkey = nk;
        c.valid = true;
    }
    std::memcpy(T, c.T, sizeof(float) * c.t.nthr);
    std::memcpy(tab, c.tab, c.t.lut_n);
    return c.t;
}

struct Bump {  // carve aligned sub-buffers out of one allocation
    char *base = nullptr;
    size_t off = 0;
    template <class T>
    T *take(size_t count)
    {
        off = (off + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
        off += sizeof(T) * std::max<size_t>(count, 1);
        return p;
    }
};

struct PinnedScratch {  // per-thread page-locked staging for results
    void *p = nullptr;
    size_t n = 0;
    ~PinnedScratch()
    {
        if (p)
            cudaFreeHost(p);
    }
    void *get(size_t bytes)
    {
        if (bytes > n) {
            if (p)
                cudaFreeHost(p);
            p = nullptr;
            n = 0;
            if (cudaHostAlloc(&p, bytes, cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
            n = bytes;
        }
        return p;
    }
};
thread_local PinnedScratch g_pinned;

struct Events {
    cudaEvent_t ev[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool ok = false;
    ~Events()
    {
        for (auto &e : ev)
            if (e)
                cudaEventDestroy(e);
    }
    bool init()
    {
        if (ok)
            return true;
        for (auto &e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                return false;
            }
        ok = true;
        return true;
    }
};
thread_local Events g_events;

void set_pool_release_threshold(int dev)
{
    static bool done[64] = {};
    if (dev < 0 || dev >= 64 || done[dev])
        return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done[dev] = true;
}

// Opt-in phase trace (environment CF_TRACE=1, diagnosis only): synchronise the
// stream at each phase boundary and print the wall time of the phase to stderr.
struct Trace {
    bool on;
    cudaStream_t st;
    double t0;
    explicit Trace(cudaStream_t s) : on(std::getenv("CF_TRACE") != nullptr), st(s), t0(now_us()) {}
    static double now_us()
    {
        return std::chrono::duration<double, std::micro>(
                   std::chrono::steady_clock::now().time_since_epoch())
            .count();
    }
    void point(const char *what)
    {
        if (!on)
            return;
        cudaStreamSynchronize(st);
        const double t = now_us();
        std::fprintf(stderr, "cf_trace %-12s %9.1f us\n", what, t - t0);
        t0 = t;
    }
};

struct Request {
    int kind;  // 0 xi, 1 rp-pi
    int autocorr;
    const cf_catalog *d1, *d2;
    std::vector<double> edges;
    double pimax;
    int npibins;
    const cf_config *cfg;
    cf_result *res;
};

int validate(const Request &q)
{
    const cf_config *c = q.cfg;
    if (!c)
        return fail(CF_EINVAL, "cfg is NULL");
    if (!q.res || !q.res->npairs)
        return fail(CF_EINVAL, "res or res->npairs is NULL");
    if (c->dtype != CF_FLOAT32 && c->dtype != CF_FLOAT64)
        return fail(CF_EINVAL, "dtype must be CF_FLOAT32 or CF_FLOAT64");
    if (c->mode != CF_MODE_FP64 && c->mode != CF_MODE_FP32_RECHECK)
        return fail(CF_EINVAL, "mode must be CF_MODE_FP64 or CF_MODE_FP32_RECHECK");
    const cf_catalog *cats[2] = {q.d1, q.autocorr ? nullptr : q.d2};
    for (int t = 0; t < 2; ++t) {
        const cf_catalog *ct = cats[t];
        if (t == 1 && q.autocorr)
            continue;
        if (!ct)
            return fail(CF_EINVAL, t ? "d2 is NULL for a cross-correlation" : "d1 is NULL");
        if (ct->n < 0 || ct->n >= (1ll << 31) - 64)
            return fail(CF_EINVAL, "catalogue size must be in [0, 2^31 - 64)");
        if (ct->n > 0 && (!ct->x || !ct->y || !ct->z))
            return fail(CF_EINVAL, "NULL coordinate array");
        if (c->weighted && ct->n > 0 && !ct->w)
            return fail(CF_EINVAL, "weighted mode needs weights for every catalogue");
    }
    if (q.edges.size() < 2)
        return fail(CF_EINVAL, "need at least 2 bin edges");
    if ((int)q.edges.size() - 1 > cf::NB_MAX)
        return fail(CF_EINVAL, "at most 64 bins");
    if (!(q.edges[0] >= 0.0) || !std::isfinite(q.edges.back()))
        return fail(CF_EINVAL, "edges must be finite and edges[0] >= 0");
    for (size_t k = 1; k < q.edges.size(); ++k)
        if (!(q.edges[k] > q.edges[k - 1]))
            return fail(CF_EINVAL, "edges must be strictly increasing");
    const double R = q.edges.back();
    if (!(R < 1e18))
        return fail(CF_EINVAL, "Rmax must be below 1e18");
    if (q.kind == 1) {
        if (!(q.pimax > 0.0) || !std::isfinite(q.pimax))
            return fail(CF_EINVAL, "pimax must be positive and finite");
        if (q.npibins < 1 || q.npibins > cf::NPI_MAX ||
            (long long)q.npibins * ((long long)q.edges.size() - 1) > cf::NBINS2D_MAX)
            return fail(CF_EINVAL, "npibins must be >= 1 with n_rp_bins * npibins <= 4096");
    }
    if (c->periodic) {
        for (int a = 0; a < 3; ++a)
            if (!(c->boxsize[a] > 0.0) || !std::isfinite(c->boxsize[a]))
                return fail(CF_EINVAL, "periodic boxsize must be positive and finite");
        const double rz = q.kind == 0 ? R : q.pimax;
        const double m = 0.5 * (1.0 - 1e-9);
        if (!(R < m * c->boxsize[0]) || !(R < m * c->boxsize[1]) || !(rz < m * c->boxsize[2]))
            return fail(CF_EINVAL, "periodic mode needs Rmax (and pimax) < boxsize/2");
    }
    for (int a = 0; a < 3; ++a)
        if (c->refine[a] < 0 || c->refine[a] > 16)
            return fail(CF_EINVAL, "refine factors must be in [0, 16]");
    if (c->pair_chunk != 0 && c->pair_chunk != 8 && c->pair_chunk != 16 && c->pair_chunk != 32)
        return fail(CF_EINVAL, "pair_chunk must be 0, 8, 16 or 32");
    if (c->pair_pp < 0 || c->pair_pp > 4 || c->pair_pp == 3)
        return fail(CF_EINVAL, "pair_pp must be 0, 1, 2 or 4");
    if (c->shard_count < 0 || (c->shard_count > 1 &&
                               (c->shard_index < 0 || c->shard_index >= c->shard_count)))
        return fail(CF_EINVAL, "shard_index must be in [0, shard_count)");
    return CF_OK;
}

// Float32 fields of the geometry used by the gridding kernels.
void finish_geom(cf::Geom &g)
{
    for (int a = 0; a < 3; ++a) {
        g.inv_wf[a] = (float)g.inv_w[a];
        long long bits = 0;
        std::memcpy(&bits, &g.box[a], 8);
        g.box_bits[a] = bits;
        g.box_bits32[a] = (int)fbits(f32_up(g.box[a]));
    }
}

// Points per column the default refinement aims at: fewer make the per-work-item
// and per-chunk costs (window records, claims, tile copies) dominate, more make
// the columns' square cross-section a poorer fit to the sphere (more pairs
// evaluated beyond Rmax).
constexpr double DEFAULT_COL_POINTS = 1024.0;

// Fewest points per column (both catalogues) the grid keeps: a sparse catalogue
// in a large box would otherwise get more columns than points, and the
// gridding and work-list costs grow with the columns.
constexpr double MIN_COL_POINTS = 32.0;

// Halve the columns on both axes until there are at most max(1, ntot /
// MIN_COL_POINTS); columns wider than Rxy / refine stay correct at any width.
void cap_columns(long long ntot, int &ncx, int &ncy)
{
    const long long cap = std::max(1ll, (long long)((double)ntot / MIN_COL_POINTS));
    while ((long long)ncx * ncy > cap && (ncx > 1 || ncy > 1)) {
        ncx = std::max(1, ncx / 2);
        ncy = std::max(1, ncy / 2);
    }
}

// Default x, y refinement (Sec. 3.1 leaves the choice to the user and names
// (2, 2, 1) as a good start): the column side s over which the smaller
// catalogue holds DEFAULT_COL_POINTS points on average (an ex x ey
// cross-section), and r = round(Rxy / s) in [1, MAX_REACH].  The smaller one
// decides because a work item's tile copies of the secondaries are spread over
// its primaries and its per-chunk costs over the secondaries in the windows;
// both want enough points per column.  Degenerate extents give 2.
int default_reach(double R, double ex, double ey, double na, double nb)
{
    const double area = ex * ey, n = std::max(std::min(na, nb), 1.0);
    if (!(area > 0.0) || !(R > 0.0) || !std::isfinite(area))
        return 2;
    const double side = std::sqrt(area * DEFAULT_COL_POINTS / n);
    return (int)std::max(1.0, std::min((double)cf::MAX_REACH, std::round(R / side)));
}

// The refinement a call uses: {0,0,0} -> (dxy, dxy, 1) with dxy the default
// x, y reach for the geometry; x, y clamped to [1, MAX_REACH], z to >= 1.
void resolve_refine(const cf_config *c, int dxy, int r[3])
{
    r[0] = c->refine[0];
    r[1] = c->refine[1];
    r[2] = c->refine[2];
    if (r[0] == 0 && r[1] == 0 && r[2] == 0) {
        r[0] = dxy;
        r[1] = dxy;
        r[2] = 1;
    }
    r[0] = std::max(1, std::min(r[0], cf::MAX_REACH));
    r[1] = std::max(1, std::min(r[1], cf::MAX_REACH));
    r[2] = std::max(1, r[2]);
}

// Catalogue sizes of a request (primaries, secondaries).
void cat_sizes(const Request &q, double &na, double &nb)
{
    na = (double)q.d1->n;
    nb = (double)(q.autocorr ? q.d1->n : q.d2->n);
}

// Grid geometry: columns of side >= Rxy / refine in x, y; z-cells for the sort.
int plan_geom(const Request &q, const double lo[3], const double hi[3], long long ntot, cf::Geom &g)
{
    const cf_config *c = q.cfg;
    const double R = q.edges.back();
    std::memset(&g, 0, sizeof(g));
    g.periodic = c->periodic ? 1 : 0;
    for (int a = 0; a < 3; ++a) {
        if (g.periodic) {
            g.origin[a] = 0.0;
            g.extent[a] = c->boxsize[a];
            g.box[a] = c->boxsize[a];
        } else {
            g.origin[a] = lo[a];
            g.extent[a] = std::max(hi[a] - lo[a], 0.0);
            g.box[a] = 0.0;
        }
    }
    double na, nb;
    cat_sizes(q, na, nb);
    int rr[3];
    resolve_refine(c, default_reach(R, g.extent[0], g.extent[1], na, nb), rr);
    const int rx = rr[0], ry = rr[1], rz = rr[2];
    g.reach_z = rz;
    auto ncol = [&](double ext, int r) {
        // Cell indices are computed in float32 (relative error <= 4 u32 per index
        // coordinate t in [0, n)): widen cells by delta >= 16 u32 n so two points
        // closer than Rmax never land more than r columns apart.
        const double nmax = std::max(1.0, std::floor(ext / R)) * r;
        const double delta = 16.0 * U32 * nmax + 1e-9;
        const double per = std::floor(ext / (R * (1.0 + delta)));
        long long n = (long long)std::max(1.0, std::min(per, 8192.0)) * r;
        return (int)std::max(1ll, n);
    };
    g.ncx = ncol(g.extent[0], rx);
    g.ncy = ncol(g.extent[1], ry);
    while ((long long)g.ncx * g.ncy > (1ll << 22)) {
        g.ncx = std::max(1, g.ncx / 2);
        g.ncy = std::max(1, g.ncy / 2);
    }
    cap_columns(ntot, g.ncx, g.ncy);
    g.ncols = g.ncx * g.ncy;
    g.reach_x = rx;
    g.reach_y = ry;
    const double per_col = (double)ntot / g.ncols;
    long long nz = (long long)std::floor(per_col * rz / 16.0);
    nz = std::max(1ll, std::min(nz, 1ll << 16));
    while (nz > 1 && (long long)g.ncols * nz > (1ll << 24) - 1)
        nz /= 2;
    g.nz = (int)nz;
    g.ncells = (long long)g.ncols * g.nz;
    const double ex = std::max(g.extent[0], 1e-300), ey = std::max(g.extent[1], 1e-300),
                 ez = std::max(g.extent[2], 1e-300);
    g.inv_w[0] = g.ncx / ex;
    g.inv_w[1] = g.ncy / ey;
    g.inv_w[2] = g.nz / ez;
    finish_geom(g);
    return CF_OK;
}

// Limit of a kernel's tile-barrier waits: 2 s (a tile copy of a few tens of KB
// that has not landed by then never will), 1 ms under CF_FLAG_DEBUG_STALL.
uint64_t wait_limit_ns(uint32_t flags)
{
    return (flags & CF_FLAG_DEBUG_STALL) ? 1000000ull : 2000000000ull;
}

// Pair-kernel parameters that depend only on the request and the geometry:
// stencil (Sec. 2.1: half stencil for auto), pruning radius and z reach
// (Sec. 2.2), float32 slacks, bins and the pi-bin error band.  M and Ls return
// the coordinate extent and the periodic shift bound of the error model.
void base_params(const Request &q, const cf::Geom &g, const cf::Gridded &A, const cf::Gridded &B,
                 cf::PairParams &P, double &M, double &Ls)
{
    const cf_config *c = q.cfg;
    const double R = q.edges.back();
    std::memset(&P, 0, sizeof(P));
    P.A = A;
    P.B = B;
    P.g = g;
    P.autocorr = q.autocorr;
    P.kind = q.kind;
    P.nstencil = 0;
    for (int ox = -g.reach_x; ox <= g.reach_x; ++ox)
        for (int oy = -g.reach_y; oy <= g.reach_y; ++oy) {
            if (q.autocorr && !(ox > 0 || (ox == 0 && oy >= 0)))
                continue;  // Sec. 2.1: each unordered column pair once
            P.stencil[P.nstencil++] = make_int2(ox, oy);
        }
    P.n_items = g.ncols * P.nstencil;
    P.shard_n = c->shard_count > 1 ? c->shard_count : 1;
    P.shard_k = c->shard_count > 1 ? c->shard_index : 0;
    P.tile_max = 1024;
    P.flags = c->flags;
    P.wait_ns = wait_limit_ns(c->flags);
    M = std::max(g.extent[0], std::max(g.extent[1], g.extent[2]));
    Ls = g.periodic ? std::max(g.box[0], std::max(g.box[1], g.box[2])) : 0.0;
    const double Rp = R * (1.0 + 1e-9) + 8.0 * U64 * (M + Ls);
    P.prune_r2 = Rp * Rp;
    P.rxy2 = Rp * Rp;
    P.rz = q.kind == 0 ? R : q.pimax;
    const double Rz = std::max(R, P.rz);
    P.zslack = (float)(8.0 * U32 * (M + Ls + Rz) + 1e-6 * Rz);
    for (int a = 0; a < 3; ++a)
        P.boxf[a] = (float)g.box[a];
    P.nbins = (int)q.edges.size() - 1;
    if (q.kind == 1) {
        P.npibins = q.npibins;
        pi_band(q.pimax, q.npibins, M, Ls, P.pscale, P.pband);
    }
}

// pi edges P_m = (pimax * m) / npibins, P_npibins = pimax (rp-pi only).
void pi_edges(const Request &q, std::vector<double> &Pe)
{
    Pe.assign(q.kind == 1 ? q.npibins + 1 : 0, 0.0);
    if (q.kind != 1)
        return;
    for (int m = 0; m < q.npibins; ++m)
        Pe[m] = (q.pimax * (double)m) / (double)q.npibins;
    Pe[q.npibins] = q.pimax;
}

int run(Request &q)
{
    int rc = validate(q);
    if (rc)
        return rc;
    const cf_config *c = q.cfg;
    cf_result *res = q.res;
    const cudaStream_t st = (cudaStream_t)c->stream;
    Trace trace(st);
    const int nb = (int)q.edges.size() - 1;
    const int nslots = q.kind == 0 ? nb : nb * q.npibins;
    const bool f64 = c->mode == CF_MODE_FP64;
    const bool wacc = c->weighted || c->want_ravg;
    const int nacc = wacc ? 2 * nslots : 0;  // binary64 wsum | rsum after the counts
    const size_t esz = c->dtype == CF_FLOAT32 ? 4 : 8;
    const cf_catalog *cats[2] = {q.d1, q.autocorr ? q.d1 : q.d2};
    const int ncat = q.autocorr ? 1 : 2;
    const double R = q.edges.back();

    std::memset(res->npairs, 0, sizeof(uint64_t) * nslots);
    if (res->wsum)
        std::memset(res->wsum, 0, sizeof(double) * nslots);
    if (res->ravg)
        std::memset(res->ravg, 0, sizeof(double) * nslots);
    res->n_cellpairs = res->n_evaluated = res->n_rechecked = res->n_band_violations = 0;
    res->kernel_ms = res->total_ms = 0.0;
    res->n_kernels = 0;
    res->refine_used[0] = res->refine_used[1] = res->refine_used[2] = 0;  // set with the grid
    res->chunk_used = c->pair_chunk ? c->pair_chunk : 16;
    res->pp_used = c->pair_pp ? c->pair_pp : 2;
    res->tuned = 0;
    res->table_linear = 0;

    int dev = 0, sms = 0;
    void *ws = nullptr, *ws2 = nullptr;
    cf::Geom g;
    cf::PairParams P;
    cf::PairLaunch PL = {};
    std::vector<double> E2(nb + 1);
    std::vector<double> Pe(q.kind == 1 ? q.npibins + 1 : 0);
    float T[2 * (cf::NB_MAX + 1)];
    uint8_t tab[cf::LUT_MAX];
    cf::Gridded G[2] = {};
    cf::GridTemps tmp = {};
    Bump bump;
    const void *dx[2][3] = {{nullptr}};
    const double *dw[2] = {nullptr, nullptr};
    bool host_in[2] = {false, false};
    long long nmax = 0, ntot = 0;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    unsigned long long *bbox_keys = nullptr;
    unsigned *d_err = nullptr, *d_ctr = nullptr, *d_wcount = nullptr;
    cf::WorkItem *work = nullptr;
    cf::Win *wins = nullptr;
    long long win_cap = 0;
    long long *wscratch = nullptr;
    unsigned long long *d_hist = nullptr, *d_diag = nullptr;
    float *d_thr = nullptr;
    uint8_t *d_lut = nullptr;
    double *d_E2 = nullptr, *d_P = nullptr;
    size_t total = 0;
    struct HostOut {
        unsigned long long hist[3 * cf::NBINS2D_MAX + 7];  // hist | diag(4) | err, counter | kept | max |w| (2) | wsum | rsum
        unsigned long long *diag;
        unsigned err;
        float thr[2 * (cf::NB_MAX + 1)];  // page-locked staging of the tables
        double e2[cf::NB_MAX + 1];
        double pe[cf::NPI_MAX + 1];
        uint8_t lut[cf::LUT_MAX];
    } *ho = nullptr;

    CF_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    CF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
    set_pool_release_threshold(dev);
    if (!g_events.init())
        return fail(CF_ECUDA, "cudaEventCreate failed");
    CF_CUDA(cudaEventRecord(g_events.ev[0], st), "cudaEventRecord");
    trace.t0 = Trace::now_us();

    for (int t = 0; t < ncat; ++t) {
        nmax = std::max<long long>(nmax, cats[t]->n);
        ntot += cats[t]->n;
        host_in[t] = cats[t]->n > 0 && !is_device_ptr(cats[t]->x);
    }
    for (int k = 0; k <= nb; ++k)
        E2[k] = q.edges[k] * q.edges[k];
    pi_edges(q, Pe);

    // Pass 1: sizes of everything except the grid (known only after the bbox).
    for (int pass = 0; pass < 2; ++pass) {
        bump.base = pass ? (char *)ws : nullptr;
        bump.off = 0;
        for (int t = 0; t < ncat; ++t) {
            const long long n = cats[t]->n;
            if (host_in[t]) {
                for (int a = 0; a < 3; ++a)
                    dx[t][a] = bump.take<char>(n * esz);
                dw[t] = cats[t]->w ? bump.take<double>(n) : nullptr;
            } else {
                dx[t][0] = cats[t]->x;
                dx[t][1] = cats[t]->y;
                dx[t][2] = cats[t]->z;
                dw[t] = cats[t]->w;
            }
        }
        bbox_keys = bump.take<unsigned long long>(6);
        // one block, one memset, one copy back: [hist | diag(4) | err, counter | wsum | rsum]
        d_hist = bump.take<unsigned long long>(nslots + 7 + nacc);
        d_diag = d_hist + nslots;
        d_err = reinterpret_cast<unsigned *>(d_hist + nslots + 4);
        d_ctr = d_err + 1;
        d_wcount = d_err + 2;
        d_thr = bump.take<float>(2 * (nb + 1));
        d_lut = bump.take<uint8_t>(cf::LUT_MAX);
        d_E2 = bump.take<double>(nb + 1);
        d_P = bump.take<double>(Pe.size());
        if (pass == 0) {
            total = bump.off;
            CF_CUDA(cudaMallocAsync(&ws, total, st), "cudaMallocAsync (inputs)");
        }
    }
    for (int t = 0; t < ncat; ++t) {
        if (!host_in[t])
            continue;
        const long long n = cats[t]->n;
        CF_CUDA(cudaMemcpyAsync((void *)dx[t][0], cats[t]->x, n * esz, cudaMemcpyHostToDevice, st), "H2D x");
        CF_CUDA(cudaMemcpyAsync((void *)dx[t][1], cats[t]->y, n * esz, cudaMemcpyHostToDevice, st), "H2D y");
        CF_CUDA(cudaMemcpyAsync((void *)dx[t][2], cats[t]->z, n * esz, cudaMemcpyHostToDevice, st), "H2D z");
        if (dw[t])
            CF_CUDA(cudaMemcpyAsync((void *)dw[t], cats[t]->w, n * 8, cudaMemcpyHostToDevice, st), "H2D w");
    }
    CF_CUDA(cudaMemsetAsync(d_hist, 0, sizeof(unsigned long long) * (nslots + 7 + nacc), st), "memset");

    ho = (HostOut *)g_pinned.get(sizeof(HostOut));
    if (!ho) {
        rc = fail(CF_ENOMEM, "cudaHostAlloc failed");
        goto cleanup;
    }

    if (!c->periodic) {  // open box: grid over the union bounding box
        unsigned long long init[6] = {~0ull, ~0ull, ~0ull, 0ull, 0ull, 0ull};
        std::memcpy(ho->hist, init, sizeof(init));
        CF_CUDA(cudaMemcpyAsync(bbox_keys, ho->hist, sizeof(init), cudaMemcpyHostToDevice, st), "H2D bbox");
        for (int t = 0; t < ncat; ++t)
            CF_CUDA(cf::launch_bbox(c->dtype, dx[t][0], dx[t][1], dx[t][2], cats[t]->n, bbox_keys, sms,
                                    d_err, st),
                    "bbox kernel");
        CF_CUDA(cudaMemcpyAsync(ho->hist, bbox_keys, sizeof(init), cudaMemcpyDeviceToHost, st), "D2H bbox");
        CF_CUDA(cudaMemcpyAsync(&ho->err, d_err, 4, cudaMemcpyDeviceToHost, st), "D2H err");
        CF_CUDA(cudaStreamSynchronize(st), "sync (bbox)");
        if (ho->err & cf::ERR_COORD) {
            rc = fail(CF_EINVAL, "non-finite coordinate");
            goto cleanup;
        }
        if (ntot > 0)
            for (int a = 0; a < 3; ++a) {
                lo[a] = cf::decode_dkey(ho->hist[a]);
                hi[a] = cf::decode_dkey(ho->hist[3 + a]);
            }
    }
    trace.point("setup");
    plan_geom(q, lo, hi, ntot, g);
    res->refine_used[0] = g.reach_x;
    res->refine_used[1] = g.reach_y;
    res->refine_used[2] = g.reach_z;

    {  // grid workspace
        // float32 mean separations: the coordinates' float32 rounding residuals,
        // unless the inputs are float32 in a periodic box (exact)
        const bool resid = !f64 && c->want_ravg && !(c->dtype == CF_FLOAT32 && c->periodic);
        for (int pass = 0; pass < 2; ++pass) {
            bump.base = pass ? (char *)ws2 : nullptr;
            bump.off = 0;
            for (int t = 0; t < ncat; ++t) {
                const long long n = cats[t]->n + 3ll * g.ncols;  // columns padded to 4
                G[t].xs = bump.take<float>(n);
                G[t].ys = bump.take<float>(n);
                G[t].zs = bump.take<float>(n);
                G[t].ws = c->weighted ? bump.take<float>(n + 64) : nullptr;  // + slack for tile reads
                if (resid) {  // float32 mean separation from inputs float32 cannot hold exactly
                    G[t].xl = bump.take<float>(n + 64);
                    G[t].yl = bump.take<float>(n + 64);
                    G[t].zl = bump.take<float>(n + 64);
                }
                G[t].wmax = c->weighted ? reinterpret_cast<unsigned *>(d_hist + nslots + 6) + t : nullptr;
                G[t].pos64 = bump.take<double4_32a>(n);
                G[t].perm = bump.take<int>(n);
                G[t].cell_start = bump.take<uint32_t>(g.ncells + 1);
                G[t].colbox = bump.take<double4_32a>(g.ncols);
            }
            tmp.cell_of = bump.take<uint32_t>(nmax);
            tmp.slot = bump.take<uint32_t>(nmax);
            tmp.tmp_idx = bump.take<int>(nmax + 3ll * g.ncols);
            tmp.tmp_key = bump.take<unsigned long long>(nmax + 3ll * g.ncols);
            tmp.counts = bump.take<uint32_t>(g.ncells + 1);
            tmp.pad = bump.take<uint32_t>(g.ncols);
            tmp.bsum = bump.take<uint32_t>(g.ncells / 4096 + 2);
            work = bump.take<cf::WorkItem>((size_t)g.ncols * cf::MAX_STENCIL);
            if (q.kind == 0 && !f64) {  // window records of the float32 DD(r) kernels
                const int sx = 2 * g.reach_x + 1, sy = 2 * g.reach_y + 1;
                const int nst = q.autocorr ? (sx * sy + 1) / 2 : sx * sy;
                const int ch = cf::xi32_chunk(c->pair_chunk ? c->pair_chunk : 16,
                                              c->pair_pp ? c->pair_pp : 2, wacc,
                                              (c->flags & CF_FLAG_VERIFY_BAND) != 0);
                win_cap = cf::win_bound(cats[0]->n, g.ncols, nst, ch);
                wins = bump.take<cf::Win>((size_t)win_cap);
            }
            // float32 weighted DD(r): 64-bit sums per thread of at most 2 CTAs per SM
            wscratch = (wacc && !f64 && q.kind == 0) ? bump.take<long long>((size_t)sms * 2 * cf::THREADS * 3 * nb)
                                                     : nullptr;
            if (pass == 0) {
                const cudaError_t e = cudaMallocAsync(&ws2, bump.off, st);
                if (e) {
                    rc = cuda_fail(e, "cudaMallocAsync (grid)");
                    goto cleanup;
                }
            }
        }
        for (int t = 0; t < ncat; ++t) {
            const cudaError_t e = cf::build_grid(c->dtype, dx[t][0], dx[t][1], dx[t][2], dw[t],
                                                 cats[t]->n, g, tmp, G[t], sms, d_err, st);
            if (e) {
                rc = cuda_fail(e, "grid kernels");
                goto cleanup;
            }
        }
        if (q.autocorr)
            G[1] = G[0];
        trace.point("gridding");

        // ---- pair kernel parameters
        double M = 0.0, Ls = 0.0;
        base_params(q, g, G[0], G[1], P, M, Ls);
        P.work = work;
        P.win = wins;
        P.win_cap = win_cap;
        P.win_count = d_err + 3;  // zeroed with the result block
        P.wscratch = wscratch;
        if (q.kind == 1) {
            std::memcpy(ho->pe, Pe.data(), 8 * Pe.size());
            CF_CUDA(cudaMemcpyAsync(d_P, ho->pe, 8 * Pe.size(), cudaMemcpyHostToDevice, st), "H2D pi edges");
        }
        if (!f64) {
            const Tables tb = cached_tables(E2.data(), nb + 1, q.kind == 0 ? 3 : 2, M, Ls, R, T, tab);
            P.nthr = tb.nthr;
            P.lut_n = tb.lut_n;
            P.lut_shift = tb.shift;
            P.u0 = tb.u0s;
            P.lut_lin = tb.lin;
            P.lut_scale = tb.lscale;
            res->table_linear = tb.lin;
            std::memcpy(ho->thr, T, 4 * P.nthr);
            std::memcpy(ho->lut, tab, P.lut_n);
            CF_CUDA(cudaMemcpyAsync(d_thr, ho->thr, 4 * P.nthr, cudaMemcpyHostToDevice, st), "H2D thresholds");
            CF_CUDA(cudaMemcpyAsync(d_lut, ho->lut, P.lut_n, cudaMemcpyHostToDevice, st), "H2D lut");
        }
        std::memcpy(ho->e2, E2.data(), 8 * E2.size());
        CF_CUDA(cudaMemcpyAsync(d_E2, ho->e2, 8 * E2.size(), cudaMemcpyHostToDevice, st), "H2D E2");
        P.thr = d_thr;
        P.lut = d_lut;
        P.E2 = d_E2;
        P.P = d_P;
        P.hist = d_hist;
        P.weighted = c->weighted ? 1 : 0;
        P.want_r = c->want_ravg ? 1 : 0;
        P.wacc = wacc ? 1 : 0;
        P.rlo = resid ? 1 : 0;
        P.wsum = wacc ? reinterpret_cast<double *>(d_hist + nslots + 7) : nullptr;
        P.rsum = wacc ? P.wsum + nslots : nullptr;
        P.diag = d_diag;
        P.err = d_err;
        P.item_counter = d_ctr;
        P.work_count = d_wcount;

        PL.f64 = f64;
        PL.chunk = c->pair_chunk ? c->pair_chunk : 16;
        PL.pp = c->pair_pp ? c->pair_pp : 2;
        PL.evals = (c->flags & (CF_FLAG_COUNT_EVALS | CF_FLAG_VERIFY_BAND)) ? 1 : 0;
        PL.verify = (!f64 && (c->flags & CF_FLAG_VERIFY_BAND)) ? 1 : 0;
        PL.max_blocks = wscratch ? sms * 2 : 0;
        PL.pipe = 1;
        cf::plan_pairs(P, PL);
        if (!f64 && PL.smem > cf::SMEM_MAX) {
            // float32 weighted rows for this many bins exceed shared memory: count
            // with the binary64 kernel instead (same results, exact per-pair terms)
            PL.f64 = 1;
            cf::plan_pairs(P, PL);
        }
        trace.point("tables");
        CF_CUDA(cudaEventRecord(g_events.ev[1], st), "cudaEventRecord");
        if (P.n_items > 0) {
            const cudaError_t e = cf::launch_pairs(P, PL, sms, st);
            if (e) {
                rc = cuda_fail(e, "pair kernel launch");
                goto cleanup;
            }
        }
        CF_CUDA(cudaEventRecord(g_events.ev[2], st), "cudaEventRecord");
        trace.point("pair kernel");
        CF_CUDA(cudaMemcpyAsync(ho->hist, d_hist, sizeof(unsigned long long) * (nslots + 7 + nacc),
                                cudaMemcpyDeviceToHost, st),
                "D2H results");
    }
    CF_CUDA(cudaEventRecord(g_events.ev[3], st), "cudaEventRecord");
    CF_CUDA(cudaEventSynchronize(g_events.ev[3]), "synchronize");
    trace.point("readback");
    {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, g_events.ev[1], g_events.ev[2]) == cudaSuccess)
            res->kernel_ms = ms;
        if (cudaEventElapsedTime(&ms, g_events.ev[0], g_events.ev[3]) == cudaSuccess)
            res->total_ms = ms;
        cudaGetLastError();
    }
    ho->diag = ho->hist + nslots;
    std::memcpy(&ho->err, ho->hist + nslots + 4, sizeof(unsigned));
    if (ho->err & cf::ERR_COORD) {
        rc = fail(CF_EINVAL, c->periodic ? "coordinate outside [0, boxsize) or non-finite"
                                         : "non-finite coordinate");
        goto cleanup;
    }
    if (ho->err & cf::ERR_TIMEOUT) {
        rc = fail(CF_ETIMEOUT, "a bounded device wait (TMA tile barrier) gave up");
        goto cleanup;
    }
    if (ho->err) {
        rc = fail(CF_EDEVICE, "kernel reported an internal inconsistency");
        goto cleanup;
    }
    {
        const uint64_t mult = q.autocorr ? 2u : 1u;  // Sec. 2.1: double the unique-pair counts
        for (int k = 0; k < nslots; ++k)
            res->npairs[k] = ho->hist[k] * mult;
        if (wacc) {
            const double *ws = reinterpret_cast<const double *>(ho->hist + nslots + 7);
            const double *rs = ws + nslots;
            for (int k = 0; k < nslots; ++k) {
                const double wk = ws[k] * (double)mult, rk = rs[k] * (double)mult;
                if (res->wsum && c->weighted)
                    res->wsum[k] = wk;
                if (res->ravg) {  // mean separation, weighted by w_i * w_j when weighted
                    const double den = c->weighted ? wk : (double)res->npairs[k];
                    res->ravg[k] = den != 0.0 ? rk / den : 0.0;
                }
            }
        }
        unsigned wcount = 0;
        std::memcpy(&wcount, reinterpret_cast<const unsigned *>(ho->hist + nslots + 4) + 2, 4);
        res->n_cellpairs = wcount;
        res->n_evaluated = ho->diag[1];
        res->n_rechecked = ho->diag[2];
        res->n_band_violations = ho->diag[3];
        for (int t = 0; t < ncat; ++t)
            res->n_kernels += cf::grid_kernels(cats[t]->n, G[t].xl != nullptr) +
                              (c->periodic ? 0 : cf::bbox_kernels(cats[t]->n));
        res->n_kernels += PL.kernels;  // work list, window pre-pass, pair kernel
    }
    rc = CF_OK;
cleanup:
    if (ws2)
        cudaFreeAsync(ws2, st);
    if (ws) {
        cudaFreeAsync(ws, st);
        if (rc == CF_OK) {
            cudaError_t e = cudaStreamSynchronize(st);
            if (e)
                rc = cuda_fail(e, "final synchronize");
        }
    }
    return rc;
}


// ---------------------------------------------------------------- autotuner
// Sec. 3.1 sweeps the refinement by hand and asks for an automatic choice: the
// tuner times a few candidates once per problem signature (the counts do not
// depend on the choice) and caches the fastest.
struct TuneChoice {
    int refine[3];
    int chunk, pp;
    double ms;
};

struct TuneCache {
    std::mutex mu;
    std::map<std::string, TuneChoice> m;
    bool env_loaded = false;
};
TuneCache g_tune;

int bucket(double v) { return (int)std::lround(2.0 * std::log2(std::max(v, 1e-3))); }

// Problem signature (half-octave buckets of the sizes and of the mean number of
// neighbours within reach).  vol: box volume (periodic) or bounding-box volume.
std::string tune_key(const Request &q, double vol)
{
    const cf_config *c = q.cfg;
    const double R = q.edges.back();
    const double n1 = (double)q.d1->n, n2 = (double)(q.autocorr ? q.d1->n : q.d2->n);
    const double reach = q.kind == 0 ? 4.0 / 3.0 * M_PI * R * R * R : M_PI * R * R * 2.0 * q.pimax;
    const double nbr = n2 * reach / std::max(vol, 1e-300);
    char buf[160];
    std::snprintf(buf, sizeof(buf), "k%d m%d d%d a%d p%d w%d n%d n%d r%d b%d", q.kind, (int)c->mode,
                  (int)c->dtype, q.autocorr, c->periodic ? 1 : 0,
                  (c->weighted || c->want_ravg) ? 1 : 0, bucket(n1), bucket(n2), bucket(nbr),
                  (int)(q.edges.size() - 1) * (q.kind == 1 ? q.npibins : 1));
    return buf;
}

int tune_save_locked(const char *path)
{
    FILE *f = std::fopen(path, "w");
    if (!f)
        return fail(CF_EINVAL, std::string("cannot write tuning cache ") + path);
    std::fprintf(f, "{\"version\": 1, \"entries\": [");
    bool first = true;
    for (const auto &kv : g_tune.m) {
        const TuneChoice &t = kv.second;
        std::fprintf(f, "%s\n {\"key\": \"%s\", \"refine\": [%d, %d, %d], \"chunk\": %d, \"pp\": %d, "
                        "\"ms\": %.6g}",
                     first ? "" : ",", kv.first.c_str(), t.refine[0], t.refine[1], t.refine[2],
                     t.chunk, t.pp, t.ms);
        first = false;
    }
    std::fprintf(f, "\n]}\n");
    return std::fclose(f) == 0 ? CF_OK : fail(CF_EINVAL, "error writing tuning cache");
}

// Parses the format tune_save_locked writes; all or nothing.
int tune_load_locked(const char *path)
{
    FILE *f = std::fopen(path, "r");
    if (!f)
        return fail(CF_EINVAL, std::string("cannot read tuning cache ") + path);
    std::string txt;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0)
        txt.append(buf, got);
    std::fclose(f);
    if (txt.find("\"version\": 1") == std::string::npos)
        return fail(CF_EINVAL, "tuning cache: missing version 1");
    std::map<std::string, TuneChoice> add;
    size_t pos = 0;
    while ((pos = txt.find("{\"key\": \"", pos)) != std::string::npos) {
        pos += 9;
        const size_t end = txt.find('"', pos);
        if (end == std::string::npos)
            return fail(CF_EINVAL, "tuning cache: unterminated key");
        const std::string key = txt.substr(pos, end - pos);
        TuneChoice t;
        if (std::sscanf(txt.c_str() + end, "\", \"refine\": [%d, %d, %d], \"chunk\": %d, \"pp\": %d, "
                                           "\"ms\": %lf}",
                        &t.refine[0], &t.refine[1], &t.refine[2], &t.chunk, &t.pp, &t.ms) != 6)
            return fail(CF_EINVAL, "tuning cache: malformed entry for key " + key);
        if (t.refine[0] < 1 || t.refine[0] > cf::MAX_REACH || t.refine[1] < 1 ||
            t.refine[1] > cf::MAX_REACH || t.refine[2] < 1 || t.refine[2] > 16 ||
            (t.chunk != 8 && t.chunk != 16 && t.chunk != 32) || (t.pp != 1 && t.pp != 2))
            return fail(CF_EINVAL, "tuning cache: out-of-range values for key " + key);
        add[key] = t;
        pos = end;
    }
    for (const auto &kv : add)
        g_tune.m[kv.first] = kv.second;
    return CF_OK;
}

void tune_env_load_locked()
{
    if (g_tune.env_loaded)
        return;
    g_tune.env_loaded = true;
    if (const char *p = std::getenv("CF_TUNE_CACHE")) {
        if (FILE *f = std::fopen(p, "r")) {
            std::fclose(f);
            const std::string keep = g_err;
            tune_load_locked(p);  // a bad file leaves the cache empty; tuning refills it
            g_err = keep;
        }
    }
}

// Volume the signature uses: the periodic box, or the bounding box of the
// inputs (one small device pass).
int tune_volume(const Request &q, double &vol)
{
    const cf_config *c = q.cfg;
    if (c->periodic) {
        vol = c->boxsize[0] * c->boxsize[1] * c->boxsize[2];
        return CF_OK;
    }
    const cudaStream_t st = (cudaStream_t)c->stream;
    const cf_catalog *cats[2] = {q.d1, q.autocorr ? q.d1 : q.d2};
    const int ncat = q.autocorr ? 1 : 2;
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
        return cuda_fail(e, "device query");
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int t = 0; t < ncat; ++t) {
        const long long n = cats[t]->n;
        if (n <= 0)
            continue;
        const void *xyz[3] = {cats[t]->x, cats[t]->y, cats[t]->z};
        if (!is_device_ptr(cats[t]->x)) {  // host inputs: scan them on the host
            for (int a = 0; a < 3; ++a)
                for (long long i = 0; i < n; ++i) {
                    const double v = c->dtype == CF_FLOAT32 ? (double)((const float *)xyz[a])[i]
                                                            : ((const double *)xyz[a])[i];
                    lo[a] = std::min(lo[a], v);
                    hi[a] = std::max(hi[a], v);
                }
            continue;
        }
        void *tmp = nullptr;
        if ((e = cudaMallocAsync(&tmp, 7 * 8, st)))
            return cuda_fail(e, "cudaMallocAsync (tuner bbox)");
        unsigned long long *keys = (unsigned long long *)tmp;
        unsigned *err = (unsigned *)(keys + 6);
        unsigned long long init[7] = {~0ull, ~0ull, ~0ull, 0ull, 0ull, 0ull, 0ull}, out[7];
        e = cudaMemcpyAsync(keys, init, sizeof(init), cudaMemcpyHostToDevice, st);
        if (!e)
            e = cf::launch_bbox(c->dtype, xyz[0], xyz[1], xyz[2], n, keys, sms, err, st);
        if (!e)
            e = cudaMemcpyAsync(out, keys, sizeof(out), cudaMemcpyDeviceToHost, st);
        if (!e)
            e = cudaStreamSynchronize(st);
        cudaFreeAsync(tmp, st);
        if (e)
            return cuda_fail(e, "tuner bbox");
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], cf::decode_dkey(out[a]));
            hi[a] = std::max(hi[a], cf::decode_dkey(out[3 + a]));
        }
    }
    vol = 1.0;
    for (int a = 0; a < 3; ++a)
        vol *= std::isfinite(hi[a] - lo[a]) ? std::max(hi[a] - lo[a], q.edges.back()) : 1.0;
    return CF_OK;
}

int run_tuned(Request &q)
{
    const cf_config *c0 = q.cfg;
    if (!c0 || !c0->autotune)
        return run(q);
    int rc = validate(q);
    if (rc)
        return rc;
    double vol = 1.0;
    if ((rc = tune_volume(q, vol)))
        return rc;
    const bool fixed_refine = c0->refine[0] || c0->refine[1] || c0->refine[2];
    std::string key = tune_key(q, vol);
    if (fixed_refine) {  // a separate entry: its choice must not reach calls that leave it open
        char buf[48];
        std::snprintf(buf, sizeof(buf), " f%d,%d,%d", c0->refine[0], c0->refine[1], c0->refine[2]);
        key += buf;
    }
    const bool shape = q.kind == 0 && c0->mode == CF_MODE_FP32_RECHECK && !c0->weighted &&
                       !c0->want_ravg && !c0->pair_chunk && !c0->pair_pp;
    TuneChoice best;
    bool have = false;
    {
        std::lock_guard<std::mutex> lock(g_tune.mu);
        tune_env_load_locked();
        auto it = g_tune.m.find(key);
        if (it != g_tune.m.end()) {
            best = it->second;
            have = true;
        }
    }
    cf_config cfg = *c0;
    cfg.autotune = 0;
    Request r = q;
    r.cfg = &cfg;
    auto apply = [&](const TuneChoice &t) {
        if (!fixed_refine)
            for (int a = 0; a < 3; ++a)
                cfg.refine[a] = t.refine[a];
        if (shape) {
            cfg.pair_chunk = t.chunk;
            cfg.pair_pp = t.pp;
        }
    };
    if (!have) {
        // candidates: the default reach for this geometry and its neighbours
        std::vector<TuneChoice> cand;
        double na, nb;
        cat_sizes(q, na, nb);
        const double ex = std::cbrt(vol), ey = ex;  // the signature's volume as a cube
        const int d = fixed_refine ? 0 : default_reach(q.edges.back(), ex, ey, na, nb);
        if (fixed_refine)  // recorded as given (clamped as the grid clamps it)
            cand.push_back(TuneChoice{{std::max(1, std::min(c0->refine[0], cf::MAX_REACH)),
                                       std::max(1, std::min(c0->refine[1], cf::MAX_REACH)),
                                       std::max(1, c0->refine[2])}, 16, 2, 0.0});
        else
            for (int rf = std::max(1, d - 1); rf <= std::min(cf::MAX_REACH, d + 1); ++rf)
                cand.push_back(TuneChoice{{rf, rf, 1}, 16, 2, 0.0});
        auto time_one = [&](TuneChoice &t, int reps) -> int {
            apply(t);
            t.ms = INFINITY;
            for (int k = 0; k < reps; ++k) {
                const int e = run(r);
                if (e)
                    return e;
                t.ms = std::min(t.ms, q.res->total_ms);
            }
            return CF_OK;
        };
        // stage 1: refinement (the first candidate once more, to absorb one-time costs)
        for (size_t k = 0; k < cand.size(); ++k)
            if ((rc = time_one(cand[k], k == 0 ? 2 : 1)))
                return rc;
        best = *std::min_element(cand.begin(), cand.end(),
                                 [](const TuneChoice &a, const TuneChoice &b) { return a.ms < b.ms; });
        // stage 2: kernel shape at that refinement
        if (shape) {
            const int shapes[3][2] = {{8, 2}, {16, 1}, {32, 1}};
            for (const auto &sh : shapes) {
                TuneChoice t = best;
                t.chunk = sh[0];
                t.pp = sh[1];
                if ((rc = time_one(t, 1)))
                    return rc;
                if (t.ms < best.ms)
                    best = t;
            }
        }
        std::lock_guard<std::mutex> lock(g_tune.mu);
        g_tune.m[key] = best;
        if (const char *p = std::getenv("CF_TUNE_CACHE")) {
            const std::string keep = g_err;
            tune_save_locked(p);
            g_err = keep;
        }
    }
    apply(best);
    rc = run(r);
    if (rc == CF_OK)
        q.res->tuned = have ? 2 : 1;
    return rc;
}
}  // namespace

extern "C" {

int cf_countpairs_xi(int autocorr, const cf_catalog *d1, const cf_catalog *d2, const double *edges,
                     int nedges, const cf_config *cfg, cf_result *res)
{
    if (!edges || nedges < 2)
        return fail(CF_EINVAL, "need at least 2 bin edges");
    Request q;
    q.kind = 0;
    q.autocorr = autocorr ? 1 : 0;
    q.d1 = d1;
    q.d2 = d2;
    q.edges.assign(edges, edges + nedges);
    q.pimax = 0.0;
    q.npibins = 0;
    q.cfg = cfg;
    q.res = res;
    return run_tuned(q);
}

int cf_countpairs_rp_pi(int autocorr, const cf_catalog *d1, const cf_catalog *d2,
                        const double *rp_edges, int n_rp_edges, double pimax, int npibins,
                        const cf_config *cfg, cf_result *res)
{
    if (!rp_edges || n_rp_edges < 2)
        return fail(CF_EINVAL, "need at least 2 rp bin edges");
    Request q;
    q.kind = 1;
    q.autocorr = autocorr ? 1 : 0;
    q.d1 = d1;
    q.d2 = d2;
    q.edges.assign(rp_edges, rp_edges + n_rp_edges);
    q.pimax = pimax;
    q.npibins = npibins;
    q.cfg = cfg;
    q.res = res;
    return run_tuned(q);
}

int cf_tune_save(const char *path)
{
    if (!path)
        return fail(CF_EINVAL, "path is NULL");
    std::lock_guard<std::mutex> lock(g_tune.mu);
    return tune_save_locked(path);
}

int cf_tune_load(const char *path)
{
    if (!path)
        return fail(CF_EINVAL, "path is NULL");
    std::lock_guard<std::mutex> lock(g_tune.mu);
    return tune_load_locked(path);
}

int cf_tune_clear(void)
{
    std::lock_guard<std::mutex> lock(g_tune.mu);
    g_tune.m.clear();
    return CF_OK;
}

int cf_tune_count(void)
{
    std::lock_guard<std::mutex> lock(g_tune.mu);
    return (int)g_tune.m.size();
}

const char *cf_last_error(void) { return g_err.c_str(); }

const char *cf_version(void) { return "cfgpu 0.1 sm_103a"; }

int cf_debug_pi_band(double pimax, int npibins, double coord_max, double shift_max,
                     float *pscale, float *pband)
{
    if (!pscale || !pband)
        return fail(CF_EINVAL, "NULL argument");
    if (!(pimax > 0.0 && std::isfinite(pimax)) || npibins < 1)
        return fail(CF_EINVAL, "pimax must be positive and finite, npibins >= 1");
    if (!(coord_max >= 0.0 && std::isfinite(coord_max)) ||
        !(shift_max >= 0.0 && std::isfinite(shift_max)))
        return fail(CF_EINVAL, "bounds must be finite and >= 0");
    pi_band(pimax, npibins, coord_max, shift_max, *pscale, *pband);
    return CF_OK;
}

static_assert(CF_BIN_TABLE_MAX == cf::LUT_MAX, "the header states the table size");

int cf_debug_bin_tables(const double *edges, int nedges, int ncomp, double coord_max,
                        double shift_max, double rmax, float *thr, unsigned char *table,
                        cf_bin_tables *info)
{
    if (!edges || !thr || !table || !info)
        return fail(CF_EINVAL, "NULL argument");
    if (nedges < 2 || nedges > cf::NB_MAX + 1)
        return fail(CF_EINVAL, "need 2 to 65 bin edges");
    for (int k = 0; k < nedges; ++k) {
        if (!std::isfinite(edges[k]) || edges[k] < 0.0)
            return fail(CF_EINVAL, "edges must be finite and >= 0");
        if (k > 0 && !(edges[k] > edges[k - 1]))
            return fail(CF_EINVAL, "edges must be strictly increasing");
    }
    if (ncomp != 2 && ncomp != 3)
        return fail(CF_EINVAL, "ncomp must be 2 or 3");
    if (!(coord_max >= 0.0 && std::isfinite(coord_max)) ||
        !(shift_max >= 0.0 && std::isfinite(shift_max)) || !(rmax >= 0.0 && std::isfinite(rmax)))
        return fail(CF_EINVAL, "bounds must be finite and >= 0");
    std::vector<double> E2(nedges);
    for (int k = 0; k < nedges; ++k)
        E2[k] = edges[k] * edges[k];
    const Tables tb = build_tables(E2.data(), nedges, ncomp, coord_max, shift_max, rmax, thr, table);
    info->nthr = tb.nthr;
    info->lut_n = tb.lut_n;
    info->lin = tb.lin;
    info->lscale = tb.lscale;
    info->shift = tb.shift;
    info->u0 = tb.u0s;
    return CF_OK;
}

}  // extern "C"

// ============================================================================
// Allocation-free DD(r): cf_countpairs_xi_noalloc.
//
// Some callers cannot allocate device memory at call time: a process whose
// device memory is already owned by another allocator (for example a
// framework's caching allocator that reserved the whole GPU), or a loop with a
// latency budget that must never wait on cudaMalloc / cudaMallocAsync.  This
// entry point runs the same gridding and pair kernels as cf_countpairs_xi, but
// every device buffer they use is carved out of one file-scope static device
// array (g_noalloc_scratch, NOALLOC_BYTES = 32 MiB), which every GPU that loads
// the library holds until the process exits.  It calls no cudaMalloc,
// cudaMallocAsync, cudaFree, cudaHostAlloc or other allocating routine, and no
// host heap allocation on its success path (tables live on the stack).
//
// The host cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so the first call on each device looks the
// address up with cudaGetSymbolAddress while that device is current, checks
// the result, and caches it; later calls reuse it.  Make that first call on a
// device before any stream capture.
//
// All calls on a device share the array and it keeps the previous call's
// contents; each call clears the counters it needs.  Two calls whose work
// overlaps on the GPU (different streams or threads without ordering) race on
// the array and give wrong results: serialise them.
// ============================================================================
namespace {

constexpr long long NOALLOC_MAX_POINTS = 1ll << 17;  // per catalogue
constexpr long long NOALLOC_MAX_CELLS = 1ll << 19;
constexpr long long NOALLOC_MAX_COLS = 1ll << 15;
constexpr size_t NOALLOC_BYTES = size_t(32) << 20;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {

std::mutex g_noalloc_mu;

// Unique id of the calling thread's current CUDA context (cuCtxGetId, reached
// through the runtime's driver entry points so the library does not link the
// driver library).  A device reset or a new context gets a new id.
typedef int (*PfnCtxGetCurrent)(void **);
typedef int (*PfnCtxGetId)(void *, unsigned long long *);

bool current_context_id(int dev, unsigned long long &id)
{
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {  // under g_noalloc_mu
        looked_up = true;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void **)&get_current, 12000,
                                             cudaEnableDefault, &q1) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess)
            get_current = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", (void **)&get_id, 12000,
                                             cudaEnableDefault, &q2) != cudaSuccess ||
            q2 != cudaDriverEntryPointSuccess)
            get_id = nullptr;
        cudaGetLastError();
    }
    if (!get_current || !get_id)
        return false;
    void *ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) {
        // no current context yet: make the device's primary context current
        if (cudaSetDevice(dev) != cudaSuccess || get_current(&ctx) != 0 || !ctx) {
            cudaGetLastError();
            return false;
        }
    }
    return get_id(ctx, &id) == 0;
}

// Device address of the static scratch in the current context.  The lookup
// (cudaGetSymbolAddress, with the device current) runs once per CUDA context:
// the first call on a device, and again after a device reset or on another
// context, since the address of a module's array belongs to its context.
struct NoallocAddr {
    unsigned long long ctx_id;
    void *ptr;
};
NoallocAddr g_noalloc_addr[64] = {};
int g_noalloc_next = 0;

int noalloc_scratch(int dev, void **out)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    unsigned long long id = 0;
    const bool have_id = current_context_id(dev, id);
    if (have_id)
        for (const NoallocAddr &a : g_noalloc_addr)
            if (a.ptr && a.ctx_id == id) {
                *out = a.ptr;
                return CF_OK;
            }
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                         "cudaGetSymbolAddress(no-alloc scratch)");
    if (have_id) {  // without a context id the lookup simply runs on every call
        g_noalloc_addr[g_noalloc_next] = NoallocAddr{id, p};
        g_noalloc_next = (g_noalloc_next + 1) % 64;
    }
    *out = p;
    return CF_OK;
}

int noalloc_xi(int autocorr, const cf_catalog *d1, const cf_catalog *d2, const double *edges,
               int nedges, const cf_config *c, cf_result *res)
{
    if (!c || !res || !res->npairs || !d1 || (!autocorr && !d2))
        return fail(CF_EINVAL, "NULL argument");
    {  // first, before any other CUDA call: the call synchronises its stream
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        const cudaError_t ec = cudaStreamIsCapturing((cudaStream_t)c->stream, &cap);
        if (ec != cudaSuccess)
            return cuda_fail(ec, "cudaStreamIsCapturing");
        if (cap != cudaStreamCaptureStatusNone)
            return fail(CF_EINVAL, "no-alloc entry point: it synchronises its stream, so it "
                                   "cannot be called while that stream is being captured");
    }
    if (!edges || nedges < 2 || nedges - 1 > cf::NB_MAX)
        return fail(CF_EINVAL, "need 2..65 bin edges");
    if (c->dtype != CF_FLOAT32 && c->dtype != CF_FLOAT64)
        return fail(CF_EINVAL, "dtype must be CF_FLOAT32 or CF_FLOAT64");
    if (c->mode != CF_MODE_FP64 && c->mode != CF_MODE_FP32_RECHECK)
        return fail(CF_EINVAL, "mode must be CF_MODE_FP64 or CF_MODE_FP32_RECHECK");
    if (c->weighted || c->want_ravg)
        return fail(CF_EINVAL, "the no-alloc entry point counts unweighted pairs only");
    if (!(edges[0] >= 0.0) || !std::isfinite(edges[nedges - 1]))
        return fail(CF_EINVAL, "edges must be finite and edges[0] >= 0");
    for (int k = 1; k < nedges; ++k)
        if (!(edges[k] > edges[k - 1]))
            return fail(CF_EINVAL, "edges must be strictly increasing");
    for (int a = 0; a < 3; ++a)
        if (c->refine[a] < 0 || c->refine[a] > 16)
            return fail(CF_EINVAL, "refine factors must be in [0, 16]");
    const cf_catalog *cats[2] = {d1, autocorr ? d1 : d2};
    const int ncat = autocorr ? 1 : 2;
    for (int t = 0; t < ncat; ++t) {
        if (cats[t]->n < 0 || cats[t]->n > NOALLOC_MAX_POINTS)
            return fail(CF_EINVAL, "no-alloc entry point: each catalogue must have at most "
                                   "131072 points (the static scratch is 32 MiB)");
        if (cats[t]->n > 0 && (!cats[t]->x || !cats[t]->y || !cats[t]->z))
            return fail(CF_EINVAL, "NULL coordinate array");
        if (cats[t]->n > 0 && (!is_device_ptr(cats[t]->x) || !is_device_ptr(cats[t]->y) ||
                               !is_device_ptr(cats[t]->z)))
            return fail(CF_EINVAL, "no-alloc entry point: coordinates must be in device memory");
    }
    const double R = edges[nedges - 1];
    if (c->periodic) {
        const double m = 0.5 * (1.0 - 1e-9);
        for (int a = 0; a < 3; ++a)
            if (!(c->boxsize[a] > 0.0) || !std::isfinite(c->boxsize[a]) || !(R < m * c->boxsize[a]))
                return fail(CF_EINVAL, "periodic mode needs a positive box and Rmax < boxsize/2");
    }
    const int nb = nedges - 1;
    const bool f64 = c->mode == CF_MODE_FP64;
    const cudaStream_t st = (cudaStream_t)c->stream;
    std::memset(res->npairs, 0, sizeof(uint64_t) * nb);
    res->n_cellpairs = res->n_evaluated = res->n_rechecked = res->n_band_violations = 0;
    res->kernel_ms = res->total_ms = 0.0;
    res->n_kernels = 0;
    res->refine_used[0] = res->refine_used[1] = res->refine_used[2] = 0;  // set with the grid
    res->chunk_used = 16;
    res->pp_used = 2;
    res->tuned = 0;
    res->table_linear = 0;

    int dev = 0, sms = 0, rc = CF_OK;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_fail(e, "device attribute");
    void *scratch = nullptr;
    if ((rc = noalloc_scratch(dev, &scratch)) != CF_OK)
        return rc;

    long long nmax = 0, ntot = 0;
    for (int t = 0; t < ncat; ++t) {
        nmax = std::max<long long>(nmax, cats[t]->n);
        ntot += cats[t]->n;
    }
    // geometry (the planner's rules, with the static-scratch caps)
    cf::Geom g;
    std::memset(&g, 0, sizeof(g));
    g.periodic = c->periodic ? 1 : 0;
    Bump bump;
    bump.base = (char *)scratch;
    unsigned long long *bbox_keys = bump.take<unsigned long long>(6);
    unsigned *d_err = bump.take<unsigned>(1);
    unsigned *d_ctr = bump.take<unsigned>(3);  // [0] item counter, [1] kept column pairs, [2] window records
    unsigned long long *d_hist = bump.take<unsigned long long>(cf::NB_MAX);
    unsigned long long *d_diag = bump.take<unsigned long long>(4);
    float *d_thr = bump.take<float>(2 * (cf::NB_MAX + 1));
    uint8_t *d_lut = bump.take<uint8_t>(cf::LUT_MAX);
    double *d_E2 = bump.take<double>(cf::NB_MAX + 1);
    struct {
        unsigned long long keys[6];
        unsigned long long hist[cf::NB_MAX];
        unsigned long long diag[4];
        unsigned err, kept;
    } h;
    if ((e = cudaMemsetAsync(d_err, 0, sizeof(unsigned), st)) != cudaSuccess)
        return cuda_fail(e, "memset");
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    if (!g.periodic) {
        const unsigned long long init[6] = {~0ull, ~0ull, ~0ull, 0ull, 0ull, 0ull};
        if ((e = cudaMemcpyAsync(bbox_keys, init, sizeof(init), cudaMemcpyHostToDevice, st)))
            return cuda_fail(e, "H2D bbox");
        for (int t = 0; t < ncat; ++t)
            if ((e = cf::launch_bbox(c->dtype, cats[t]->x, cats[t]->y, cats[t]->z, cats[t]->n,
                                     bbox_keys, sms, d_err, st)))
                return cuda_fail(e, "bbox kernel");
        if ((e = cudaMemcpyAsync(h.keys, bbox_keys, sizeof(h.keys), cudaMemcpyDeviceToHost, st)) ||
            (e = cudaMemcpyAsync(&h.err, d_err, 4, cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st)))
            return cuda_fail(e, "bbox readback");
        if (h.err & cf::ERR_COORD)
            return fail(CF_EINVAL, "non-finite coordinate");
        if (ntot > 0)
            for (int a = 0; a < 3; ++a) {
                lo[a] = cf::decode_dkey(h.keys[a]);
                hi[a] = cf::decode_dkey(h.keys[3 + a]);
            }
    }
    for (int a = 0; a < 3; ++a) {
        g.origin[a] = g.periodic ? 0.0 : lo[a];
        g.extent[a] = g.periodic ? c->boxsize[a] : std::max(hi[a] - lo[a], 0.0);
        g.box[a] = g.periodic ? c->boxsize[a] : 0.0;
    }
    int rr[3];
    resolve_refine(c, default_reach(R, g.extent[0], g.extent[1], (double)d1->n,
                                    (double)(autocorr ? d1->n : d2->n)), rr);
    const int rx = rr[0], ry = rr[1], rz = rr[2];
    g.reach_z = rz;
    auto ncol = [&](double ext, int r) {  // same rule as plan_geom
        const double nmax = std::max(1.0, std::floor(ext / R)) * r;
        const double delta = 16.0 * U32 * nmax + 1e-9;
        const double per = std::floor(ext / (R * (1.0 + delta)));
        return (int)std::max(1ll, (long long)std::max(1.0, std::min(per, 8192.0)) * r);
    };
    // z-cells of the in-column sort for a given column count (plan_geom's rule)
    auto zcells = [&](long long ncols) {
        long long nz = (long long)std::floor((double)ntot / ncols * rz / 16.0);
        nz = std::max(1ll, std::min(nz, 1ll << 16));
        while (nz > 1 && ncols * nz > NOALLOC_MAX_CELLS)
            nz /= 2;
        return nz;
    };
    g.ncx = ncol(g.extent[0], rx);
    g.ncy = ncol(g.extent[1], ry);
    cap_columns(ntot, g.ncx, g.ncy);
    while ((long long)g.ncx * g.ncy > NOALLOC_MAX_COLS) {  // wider columns stay correct
        g.ncx = std::max(1, g.ncx / 2);
        g.ncy = std::max(1, g.ncy / 2);
    }
    g.nz = (int)zcells((long long)g.ncx * g.ncy);
    g.reach_x = rx;
    g.reach_y = ry;
    res->refine_used[0] = rx;
    res->refine_used[1] = ry;
    res->refine_used[2] = rz;
    const int nstencil_max = autocorr ? ((2 * g.reach_x + 1) * (2 * g.reach_y + 1) + 1) / 2
                                      : (2 * g.reach_x + 1) * (2 * g.reach_y + 1);
    cf::Gridded G[2] = {};
    cf::GridTemps tmp = {};
    cf::WorkItem *work = nullptr;
    cf::Win *wins = nullptr;
    long long win_cap = 0;
    const int win_ch = cf::xi32_chunk(16, 2, false, false);  // the kernel shape of this entry point
    // Carve the grids, temporaries and the work list for the current geometry
    // out of the array; if they do not fit, plan coarser (columns at least
    // Rmax / refine wide stay correct at any width, and fewer z-cells only make
    // the in-column sort work harder) and try again.
    for (;;) {
        g.ncols = g.ncx * g.ncy;
        g.ncells = (long long)g.ncols * g.nz;
        Bump b = bump;
        for (int t = 0; t < ncat; ++t) {
            const long long n = cats[t]->n + 3ll * g.ncols;  // columns padded to 4
            G[t] = cf::Gridded{};
            G[t].xs = b.take<float>(n);
            G[t].ys = b.take<float>(n);
            G[t].zs = b.take<float>(n);
            G[t].pos64 = b.take<double4_32a>(n);
            G[t].perm = b.take<int>(n);
            G[t].cell_start = b.take<uint32_t>(g.ncells + 1);
            G[t].colbox = b.take<double4_32a>(g.ncols);
        }
        tmp.cell_of = b.take<uint32_t>(nmax);
        tmp.slot = b.take<uint32_t>(nmax);
        tmp.tmp_idx = b.take<int>(nmax + 3ll * g.ncols);
        tmp.tmp_key = b.take<unsigned long long>(nmax + 3ll * g.ncols);
        tmp.counts = b.take<uint32_t>(g.ncells + 1);
        tmp.pad = b.take<uint32_t>(g.ncols);
        tmp.bsum = b.take<uint32_t>(g.ncells / 4096 + 2);
        work = b.take<cf::WorkItem>((size_t)g.ncols * nstencil_max);
        win_cap = f64 ? 0 : cf::win_bound(cats[0]->n, g.ncols, nstencil_max, win_ch);
        wins = f64 ? nullptr : b.take<cf::Win>((size_t)win_cap);
        if (b.off <= NOALLOC_BYTES) {
            bump = b;
            break;
        }
        if (g.ncx > 1 || g.ncy > 1) {
            g.ncx = std::max(1, g.ncx / 2);
            g.ncy = std::max(1, g.ncy / 2);
            g.nz = (int)zcells((long long)g.ncx * g.ncy);
        } else if (g.nz > 1) {
            g.nz /= 2;
        } else {
            return fail(CF_EINVAL, "no-alloc entry point: problem does not fit the 32 MiB static scratch");
        }
    }
    g.inv_w[0] = g.ncx / std::max(g.extent[0], 1e-300);
    g.inv_w[1] = g.ncy / std::max(g.extent[1], 1e-300);
    g.inv_w[2] = g.nz / std::max(g.extent[2], 1e-300);
    finish_geom(g);

    if ((e = cudaMemsetAsync(d_ctr, 0, 3 * sizeof(unsigned), st)) ||
        (e = cudaMemsetAsync(d_hist, 0, sizeof(unsigned long long) * nb, st)) ||
        (e = cudaMemsetAsync(d_diag, 0, sizeof(unsigned long long) * 4, st)))
        return cuda_fail(e, "memset");
    for (int t = 0; t < ncat; ++t)
        if ((e = cf::build_grid(c->dtype, cats[t]->x, cats[t]->y, cats[t]->z, nullptr, cats[t]->n,
                                g, tmp, G[t], sms, d_err, st)))
            return cuda_fail(e, "grid kernels");
    if (autocorr)
        G[1] = G[0];

    double E2[cf::NB_MAX + 1];
    for (int k = 0; k <= nb; ++k)
        E2[k] = edges[k] * edges[k];
    cf::PairParams P;
    std::memset(&P, 0, sizeof(P));
    P.A = G[0];
    P.B = G[1];
    P.g = g;
    P.autocorr = autocorr ? 1 : 0;
    P.kind = 0;
    for (int ox = -g.reach_x; ox <= g.reach_x; ++ox)
        for (int oy = -g.reach_y; oy <= g.reach_y; ++oy) {
            if (autocorr && !(ox > 0 || (ox == 0 && oy >= 0)))
                continue;
            P.stencil[P.nstencil++] = make_int2(ox, oy);
        }
    P.n_items = g.ncols * P.nstencil;
    P.work = work;
    P.work_count = d_ctr + 1;
    P.win = wins;
    P.win_cap = win_cap;
    P.win_count = d_ctr + 2;
    P.tile_max = 1024;
    P.flags = c->flags & (CF_FLAG_NO_PRUNE | CF_FLAG_COUNT_EVALS);
    P.wait_ns = wait_limit_ns(P.flags);
    const double M = std::max(g.extent[0], std::max(g.extent[1], g.extent[2]));
    const double Ls = g.periodic ? std::max(g.box[0], std::max(g.box[1], g.box[2])) : 0.0;
    const double Rp = R * (1.0 + 1e-9) + 8.0 * U64 * (M + Ls);
    P.prune_r2 = Rp * Rp;
    P.rxy2 = Rp * Rp;
    P.rz = R;
    P.zslack = (float)(8.0 * U32 * (M + Ls + R) + 1e-6 * R);
    for (int a = 0; a < 3; ++a)
        P.boxf[a] = (float)g.box[a];
    P.nbins = nb;
    float T[2 * (cf::NB_MAX + 1)];
    uint8_t tab[cf::LUT_MAX];
    if (!f64) {
        const Tables tb = cached_tables(E2, nb + 1, 3, M, Ls, R, T, tab);
        P.nthr = tb.nthr;
        P.lut_n = tb.lut_n;
        P.lut_shift = tb.shift;
        P.u0 = tb.u0s;
        P.lut_lin = tb.lin;
        P.lut_scale = tb.lscale;
        res->table_linear = tb.lin;
        if ((e = cudaMemcpyAsync(d_thr, T, sizeof(float) * P.nthr, cudaMemcpyHostToDevice, st)) ||
            (e = cudaMemcpyAsync(d_lut, tab, P.lut_n, cudaMemcpyHostToDevice, st)))
            return cuda_fail(e, "H2D tables");
    }
    if ((e = cudaMemcpyAsync(d_E2, E2, sizeof(double) * (nb + 1), cudaMemcpyHostToDevice, st)))
        return cuda_fail(e, "H2D E2");
    P.thr = d_thr;
    P.lut = d_lut;
    P.E2 = d_E2;
    P.hist = d_hist;
    P.diag = d_diag;
    P.err = d_err;
    P.item_counter = d_ctr;
    cf::PairLaunch PL;
    std::memset(&PL, 0, sizeof(PL));
    PL.f64 = f64;
    PL.chunk = 16;
    PL.pp = 2;
    PL.evals = (P.flags & CF_FLAG_COUNT_EVALS) ? 1 : 0;
    PL.pipe = 1;
    cf::plan_pairs(P, PL);
    if (P.n_items > 0 && (e = cf::launch_pairs(P, PL, sms, st)))
        return cuda_fail(e, "pair kernel launch");
    if ((e = cudaMemcpyAsync(h.hist, d_hist, sizeof(unsigned long long) * nb, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaMemcpyAsync(h.diag, d_diag, sizeof(h.diag), cudaMemcpyDeviceToHost, st)) ||
        (e = cudaMemcpyAsync(&h.kept, d_ctr + 1, 4, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaMemcpyAsync(&h.err, d_err, 4, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st)))
        return cuda_fail(e, "result readback");
    if (h.err & cf::ERR_COORD)
        return fail(CF_EINVAL, "coordinate outside [0, boxsize) or non-finite");
    if (h.err & cf::ERR_TIMEOUT)
        return fail(CF_ETIMEOUT, "a bounded device wait (TMA tile barrier) gave up");
    if (h.err)
        return fail(CF_EDEVICE, "kernel reported an internal inconsistency");
    const uint64_t mult = autocorr ? 2u : 1u;
    for (int k = 0; k < nb; ++k)
        res->npairs[k] = h.hist[k] * mult;
    res->n_cellpairs = h.kept;
    res->n_evaluated = h.diag[1];
    res->n_rechecked = h.diag[2];
    for (int t = 0; t < ncat; ++t)
        res->n_kernels += cf::grid_kernels(cats[t]->n) + (c->periodic ? 0 : cf::bbox_kernels(cats[t]->n));
    res->n_kernels += PL.kernels;  // work list, window pre-pass, pair kernel
    return CF_OK;
}

}  // namespace

extern "C" int cf_countpairs_xi_noalloc(int autocorr, const cf_catalog *d1, const cf_catalog *d2,
                                        const double *edges, int nedges, const cf_config *cfg,
                                        cf_result *res)
{
    return noalloc_xi(autocorr ? 1 : 0, d1, d2, edges, nedges, cfg, res);
}

// ============================================================================
// Batched counting: cf_batch_*.
// ============================================================================
namespace {


struct BatchJob {
    Request q;
    cf_catalog cat[2];
    cf_config cfg;
    std::vector<double> edges;
    int ncat = 1;
    // plan
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    cf::Geom g;
    cf::Gridded G[2] = {};
    cf::PairParams P;
    int path = 0, nslots = 0, smem = 0;
    int chunk = 16, pp = 2;  // float32 DD(r) kernel shape (tuned or the default 16 x 2)
    int tuned = 0;           // as cf_result.tuned: 1 tuned at plan time, 2 cached choice used
    size_t out_off = 0;  // u64 words into the output block: [hist | diag(4) | err, - | kept, -]
    uint64_t n_kernels = 0;
};

}  // namespace

struct cf_batch {
    std::vector<BatchJob> jobs;
    bool planned = false;
    int dev = -1, sms = 0, smem_max = 0, blocks = 0;
    void *ws = nullptr;                  // one device workspace for every job
    unsigned long long *d_out = nullptr; // output block (all jobs)
    size_t out_words = 0;
    unsigned long long *h_out = nullptr; // page-locked copy of the output block
    cf::PairParams *d_jobs = nullptr;
    int *d_path = nullptr;
    unsigned *d_offsets = nullptr, *d_counter = nullptr;
    unsigned long long *d_bbox = nullptr;
    cf::GridBatch grid = {};             // every catalogue of every job, gridded in one pass
    unsigned *d_wpre = nullptr;          // work-list blocks: prefix over the jobs
    unsigned wblocks = 0;
    cudaStream_t own = nullptr;
    cudaEvent_t ev[4] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    uint64_t n_kernels = 0;
};

namespace {

void batch_free_plan(cf_batch *b)
{
    if (b->gexec)
        cudaGraphExecDestroy(b->gexec);
    if (b->graph)
        cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    if (b->ws)
        cudaFree(b->ws);
    if (b->h_out)
        cudaFreeHost(b->h_out);
    b->ws = nullptr;
    b->h_out = nullptr;
    b->planned = false;
    cudaGetLastError();
}

int batch_add(cf_batch *b, Request &q)
{
    if (!b)
        return fail(CF_EINVAL, "batch is NULL");
    if ((int)b->jobs.size() >= cf::BATCH_MAX)
        return fail(CF_EINVAL, "a batch holds at most 1024 jobs");
    int rc = validate(q);
    if (rc)
        return rc;
    if (q.cfg->weighted || q.cfg->want_ravg)
        return fail(CF_EINVAL, "batched jobs count unweighted pairs (no weights, no ravg)");
    const cf_catalog *cats[2] = {q.d1, q.autocorr ? q.d1 : q.d2};
    for (int t = 0; t < (q.autocorr ? 1 : 2); ++t)
        if (cats[t]->n > 0 && (!is_device_ptr(cats[t]->x) || !is_device_ptr(cats[t]->y) ||
                               !is_device_ptr(cats[t]->z)))
            return fail(CF_EINVAL, "batched jobs take coordinates in device memory");
    BatchJob j;
    j.cat[0] = *q.d1;
    if (!q.autocorr)
        j.cat[1] = *q.d2;
    j.cfg = *q.cfg;
    j.edges = q.edges;
    j.ncat = q.autocorr ? 1 : 2;
    j.q = q;
    b->jobs.push_back(j);
    b->planned = false;  // a new job invalidates the plan and the graph
    return CF_OK;
}

// Request of job k with its pointers into the job's own copies.
void batch_bind(BatchJob &j)
{
    j.q.d1 = &j.cat[0];
    j.q.d2 = j.q.autocorr ? nullptr : &j.cat[1];
    j.q.cfg = &j.cfg;
    j.q.edges = j.edges;
}

// Bounding boxes of every open-box job (one pass, one synchronisation).
int batch_bboxes(cf_batch *b, cudaStream_t st, std::vector<std::array<double, 6>> &box)
{
    const int nj = (int)b->jobs.size();
    box.assign(nj, {0, 0, 0, 0, 0, 0});
    int nopen = 0;
    for (auto &j : b->jobs)
        nopen += j.cfg.periodic ? 0 : 1;
    if (!nopen)
        return CF_OK;
    unsigned long long *keys = nullptr;
    const size_t words = (size_t)nj * 2 * 7;
    cudaError_t e = cudaMallocAsync(&keys, words * 8, st);
    if (e)
        return cuda_fail(e, "cudaMallocAsync (batch bbox)");
    std::vector<unsigned long long> h(words, 0ull);
    for (int k = 0; k < nj * 2; ++k)
        for (int a = 0; a < 3; ++a)
            h[k * 7 + a] = ~0ull;
    e = cudaMemcpyAsync(keys, h.data(), words * 8, cudaMemcpyHostToDevice, st);
    for (int k = 0; k < nj && !e; ++k) {
        BatchJob &j = b->jobs[k];
        if (j.cfg.periodic)
            continue;
        for (int t = 0; t < j.ncat && !e; ++t)
            e = cf::launch_bbox(j.cfg.dtype, j.cat[t].x, j.cat[t].y, j.cat[t].z, j.cat[t].n,
                                keys + (k * 2 + t) * 7, b->sms,
                                reinterpret_cast<unsigned *>(keys + (k * 2 + t) * 7 + 6), st);
    }
    if (!e)
        e = cudaMemcpyAsync(h.data(), keys, words * 8, cudaMemcpyDeviceToHost, st);
    if (!e)
        e = cudaStreamSynchronize(st);
    cudaFreeAsync(keys, st);
    if (e)
        return cuda_fail(e, "batch bounding boxes");
    for (int k = 0; k < nj; ++k) {
        BatchJob &j = b->jobs[k];
        if (j.cfg.periodic)
            continue;
        double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        bool any = false;
        for (int t = 0; t < j.ncat; ++t) {
            const unsigned long long *kk = h.data() + (k * 2 + t) * 7;
            if (reinterpret_cast<const unsigned *>(kk + 6)[0] & cf::ERR_COORD)
                return fail(CF_EINVAL, "batch job " + std::to_string(k) + ": non-finite coordinate");
            if (j.cat[t].n <= 0)
                continue;
            for (int a = 0; a < 3; ++a) {
                const double l = cf::decode_dkey(kk[a]), u = cf::decode_dkey(kk[3 + a]);
                lo[a] = any ? std::min(lo[a], l) : l;
                hi[a] = any ? std::max(hi[a], u) : u;
            }
            any = true;
        }
        box[k] = {lo[0], lo[1], lo[2], hi[0], hi[1], hi[2]};
    }
    return CF_OK;
}

int batch_plan(cf_batch *b, cudaStream_t st, const std::vector<std::array<double, 6>> &box)
{
    batch_free_plan(b);
    const int nj = (int)b->jobs.size();
    // refinement and float32 DD(r) kernel shape: with autotune the tuner's choice
    // for the job's signature (Sec. 3.1), timed now with single calls when the
    // cache has none; else the job's own refinement and the default shape
    for (int k = 0; k < nj; ++k) {
        BatchJob &j = b->jobs[k];
        batch_bind(j);
        for (int a = 0; a < 3; ++a) {
            j.lo[a] = box[k][a];
            j.hi[a] = box[k][3 + a];
        }
        j.chunk = 16;
        j.pp = 2;
        j.tuned = 0;
        if (j.cfg.autotune) {
            const bool fixed_refine = j.cfg.refine[0] || j.cfg.refine[1] || j.cfg.refine[2];
            double vol = 1.0;
            for (int a = 0; a < 3; ++a)
                vol *= j.cfg.periodic ? j.cfg.boxsize[a] : std::max(j.hi[a] - j.lo[a], j.edges.back());
            const std::string key = tune_key(j.q, vol);
            TuneChoice ch;
            bool have = false;
            auto lookup = [&]() {
                std::lock_guard<std::mutex> lock(g_tune.mu);
                tune_env_load_locked();
                auto it = g_tune.m.find(key);
                if (it != g_tune.m.end()) {
                    ch = it->second;
                    have = true;
                }
            };
            lookup();
            j.tuned = have ? 2 : 1;
            if (!have) {  // time the candidates with single calls, as cf_countpairs_xi does
                const int ns = j.q.kind == 0 ? (int)j.edges.size() - 1
                                              : ((int)j.edges.size() - 1) * j.q.npibins;
                std::vector<uint64_t> scratch(ns);
                cf_result tr;
                std::memset(&tr, 0, sizeof(tr));
                tr.npairs = scratch.data();
                Request r = j.q;
                r.res = &tr;
                const int rc = run_tuned(r);
                if (rc)
                    return fail(rc, "batch job " + std::to_string(k) + " autotuning: " + g_err);
                lookup();
            }
            if (have) {
                if (!fixed_refine)
                    for (int a = 0; a < 3; ++a)
                        j.cfg.refine[a] = ch.refine[a];
                if (j.q.kind == 0 && j.cfg.mode == CF_MODE_FP32_RECHECK) {
                    j.chunk = ch.chunk;
                    j.pp = ch.pp;
                }
            }
        }
        long long ntot = 0;
        for (int t = 0; t < j.ncat; ++t)
            ntot += j.cat[t].n;
        plan_geom(j.q, j.lo, j.hi, ntot, j.g);
        j.nslots = j.q.kind == 0 ? (int)j.edges.size() - 1 : ((int)j.edges.size() - 1) * j.q.npibins;
    }
    // sizes, then the workspace, then pointers (two passes of the same carving)
    std::vector<std::vector<float>> T(nj);
    std::vector<std::vector<uint8_t>> tab(nj);
    std::vector<Tables> tb(nj);
    std::vector<std::vector<double>> E2(nj), Pe(nj);
    size_t out_words = 0;
    for (int k = 0; k < nj; ++k) {
        b->jobs[k].out_off = out_words;
        out_words += (size_t)b->jobs[k].nslots + 8;
    }
    // one gridding segment per catalogue of every job; its entries in the
    // concatenated per-cell arrays start at c0 (ncells + 1 each)
    std::vector<cf::GridSeg> seg;
    long long ctot = 0;
    for (int k = 0; k < nj; ++k) {
        const BatchJob &j = b->jobs[k];
        for (int t = 0; t < j.ncat; ++t) {
            cf::GridSeg sg;
            std::memset(&sg, 0, sizeof(sg));
            sg.x = j.cat[t].x;
            sg.y = j.cat[t].y;
            sg.z = j.cat[t].z;
            sg.f32 = j.cfg.dtype == CF_FLOAT32 ? 1 : 0;
            sg.job = k;
            sg.n = j.cat[t].n;
            sg.c0 = ctot;
            ctot += j.g.ncells + 1;
            seg.push_back(sg);
        }
    }
    const int nseg = (int)seg.size();
    std::vector<unsigned> pre[cf::GB_SHAPES], wpre(nj + 1, 0u);
    for (int k = 0; k < cf::GB_SHAPES; ++k) {
        pre[k].assign(nseg + 1, 0u);
        for (int q = 0; q < nseg; ++q)
            pre[k][q + 1] = pre[k][q] + cf::grid_batch_blocks(k, seg[q].n, b->jobs[seg[q].job].g);
    }
    Bump bump;
    cudaError_t e;
    for (int pass = 0; pass < 2; ++pass) {
        bump.base = pass ? (char *)b->ws : nullptr;
        bump.off = 0;
        b->d_out = bump.take<unsigned long long>(out_words);
        b->d_jobs = bump.take<cf::PairParams>(nj);
        b->d_path = bump.take<int>(nj);
        b->d_offsets = bump.take<unsigned>(nj + 1);
        b->d_counter = bump.take<unsigned>(1);
        cf::GridBatch &gb = b->grid;
        gb.seg = bump.take<cf::GridSeg>(nseg);
        gb.geom = bump.take<cf::Geom>(nj);
        gb.nseg = nseg;
        gb.ctot = ctot;
        gb.counts = bump.take<uint32_t>(ctot + 1);
        gb.scan = bump.take<uint32_t>(ctot);
        gb.bsum = bump.take<uint32_t>(cf::scan_block_sums(ctot));
        for (int k = 0; k < cf::GB_SHAPES; ++k) {
            gb.pre[k] = bump.take<unsigned>(nseg + 1);
            gb.blocks[k] = pre[k][nseg];
        }
        b->d_wpre = bump.take<unsigned>(nj + 1);
        int q = 0;
        for (int k = 0; k < nj; ++k) {
            BatchJob &j = b->jobs[k];
            for (int t = 0; t < j.ncat; ++t, ++q) {
                const long long n = j.cat[t].n + 3ll * j.g.ncols;
                cf::Gridded &G = j.G[t];
                G.n = j.cat[t].n;
                G.xs = bump.take<float>(n);
                G.ys = bump.take<float>(n);
                G.zs = bump.take<float>(n);
                G.ws = nullptr;
                G.pos64 = bump.take<double4_32a>(n);
                G.perm = bump.take<int>(n);
                G.cell_start = bump.take<uint32_t>(j.g.ncells + 1);
                G.colbox = bump.take<double4_32a>(j.g.ncols);
                cf::GridSeg &sg = seg[q];
                sg.out = G;
                sg.cell_of = bump.take<uint32_t>(j.cat[t].n);
                sg.slot = bump.take<uint32_t>(j.cat[t].n);
                sg.tmp_idx = bump.take<int>(n);
                sg.tmp_key = bump.take<unsigned long long>(n);
                sg.pad = bump.take<uint32_t>(j.g.ncols);
            }
            if (j.ncat == 1)
                j.G[1] = j.G[0];
            const int nb = (int)j.edges.size() - 1;
            j.P.work = bump.take<cf::WorkItem>((size_t)j.g.ncols * cf::MAX_STENCIL);
            j.P.thr = bump.take<float>(2 * (nb + 1));
            j.P.lut = bump.take<uint8_t>(cf::LUT_MAX);
            j.P.E2 = bump.take<double>(nb + 1);
            j.P.P = bump.take<double>(j.q.kind == 1 ? j.q.npibins + 1 : 1);
        }
        if (pass == 0) {
            if ((e = cudaMalloc(&b->ws, bump.off)))
                return cuda_fail(e, "cudaMalloc (batch workspace)");
        }
    }
    if ((e = cudaHostAlloc((void **)&b->h_out, out_words * 8, cudaHostAllocDefault)))
        return cuda_fail(e, "cudaHostAlloc (batch results)");
    b->out_words = out_words;
    // parameters and tables of every job
    std::vector<cf::PairParams> hp(nj);
    std::vector<int> hpath(nj);
    b->smem_max = 0;
    for (int k = 0; k < nj; ++k) {
        BatchJob &j = b->jobs[k];
        const int nb = (int)j.edges.size() - 1;
        const bool f64 = j.cfg.mode == CF_MODE_FP64;
        cf::WorkItem *work = j.P.work;
        const float *dthr = j.P.thr;
        const uint8_t *dlut = j.P.lut;
        const double *dE2 = j.P.E2, *dP = j.P.P;
        double M = 0.0, Ls = 0.0;
        base_params(j.q, j.g, j.G[0], j.G[1], j.P, M, Ls);
        j.P.flags = j.cfg.flags & CF_FLAG_NO_PRUNE;
        j.P.work = work;
        j.P.thr = dthr;
        j.P.lut = dlut;
        j.P.E2 = dE2;
        j.P.P = dP;
        E2[k].resize(nb + 1);
        for (int q = 0; q <= nb; ++q)
            E2[k][q] = j.edges[q] * j.edges[q];
        pi_edges(j.q, Pe[k]);
        if (!f64) {
            T[k].resize(2 * (nb + 1));
            tab[k].resize(cf::LUT_MAX);
            tb[k] = build_tables(E2[k].data(), nb + 1, j.q.kind == 0 ? 3 : 2, M, Ls, j.edges.back(),
                                 T[k].data(), tab[k].data());
            j.P.nthr = tb[k].nthr;
            j.P.lut_n = tb[k].lut_n;
            j.P.lut_shift = tb[k].shift;
            j.P.u0 = tb[k].u0s;
            j.P.lut_lin = tb[k].lin;
            j.P.lut_scale = tb[k].lscale;
            if ((e = cudaMemcpy((void *)dthr, T[k].data(), 4 * j.P.nthr, cudaMemcpyHostToDevice)) ||
                (e = cudaMemcpy((void *)dlut, tab[k].data(), j.P.lut_n, cudaMemcpyHostToDevice)))
                return cuda_fail(e, "H2D batch tables");
        }
        if ((e = cudaMemcpy((void *)dE2, E2[k].data(), 8 * (nb + 1), cudaMemcpyHostToDevice)))
            return cuda_fail(e, "H2D batch edges");
        if (j.q.kind == 1 &&
            (e = cudaMemcpy((void *)dP, Pe[k].data(), 8 * Pe[k].size(), cudaMemcpyHostToDevice)))
            return cuda_fail(e, "H2D batch pi edges");
        unsigned long long *o = b->d_out + j.out_off;
        j.P.hist = o;
        j.P.diag = o + j.nslots;
        j.P.err = reinterpret_cast<unsigned *>(o + j.nslots + 4);
        j.P.item_counter = j.P.err + 1;
        j.P.work_count = j.P.err + 2;
        cf::PairLaunch PL;
        std::memset(&PL, 0, sizeof(PL));
        PL.f64 = f64;
        PL.chunk = j.chunk;
        PL.pp = j.pp;
        cf::plan_pairs(j.P, PL);
        j.smem = PL.smem;
        j.path = cf::batch_path(j.P, f64, j.chunk, j.pp);
        b->smem_max = std::max(b->smem_max, PL.smem);
        hp[k] = j.P;
        hpath[k] = j.path;
        j.n_kernels = 0;  // the batch's launches are shared by all jobs (batch statistics)
        wpre[k + 1] = wpre[k] + (unsigned)((std::max(j.P.n_items, 0) + 255) / 256);
    }
    for (auto &sg : seg)
        sg.err = b->jobs[sg.job].P.err;
    std::vector<cf::Geom> geom(nj);
    for (int k = 0; k < nj; ++k)
        geom[k] = b->jobs[k].g;
    b->wblocks = wpre[nj];
    if ((e = cudaMemcpy(b->d_jobs, hp.data(), sizeof(cf::PairParams) * nj, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->d_path, hpath.data(), sizeof(int) * nj, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy((void *)b->grid.seg, seg.data(), sizeof(cf::GridSeg) * nseg, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy((void *)b->grid.geom, geom.data(), sizeof(cf::Geom) * nj, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->d_wpre, wpre.data(), sizeof(unsigned) * (nj + 1), cudaMemcpyHostToDevice)))
        return cuda_fail(e, "H2D batch jobs");
    for (int k = 0; k < cf::GB_SHAPES; ++k)
        if ((e = cudaMemcpy((void *)b->grid.pre[k], pre[k].data(), sizeof(unsigned) * (nseg + 1),
                            cudaMemcpyHostToDevice)))
            return cuda_fail(e, "H2D batch gridding plan");
    // two memsets, the batched gridding, the work lists, offsets + batched pair kernel
    b->n_kernels = 2 + cf::grid_batch_kernels() + 1 + 2;
    b->planned = true;
    (void)st;
    return CF_OK;
}

// The whole device sequence of one run, on stream st (captured or direct;
// timing events are recorded only when not capturing).
int batch_issue(cf_batch *b, cudaStream_t st, bool capturing)
{
    cudaError_t e;
    const int nj = (int)b->jobs.size();
    if ((!capturing && (e = cudaEventRecord(b->ev[0], st))) ||
        (e = cudaMemsetAsync(b->d_out, 0, b->out_words * 8, st)) ||
        (e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned), st)))
        return cuda_fail(e, "batch start");
    // every catalogue of every job gridded stage by stage, then every work list
    if ((e = cf::build_grid_batch(b->grid, b->sms, st)))
        return cuda_fail(e, "batched gridding");
    if ((e = cf::launch_worklist_batch(b->d_jobs, b->d_wpre, nj, b->wblocks, st)))
        return cuda_fail(e, "batched work lists");
    cf::BatchParams B;
    B.jobs = b->d_jobs;
    B.path = b->d_path;
    B.njobs = nj;
    B.offsets = b->d_offsets;
    B.item_counter = b->d_counter;
    if ((!capturing && (e = cudaEventRecord(b->ev[1], st))) ||
        (e = cf::launch_batch(B, b->smem_max, b->sms, b->blocks, st)) ||
        (!capturing && (e = cudaEventRecord(b->ev[2], st))) ||
        (e = cudaMemcpyAsync(b->h_out, b->d_out, b->out_words * 8, cudaMemcpyDeviceToHost, st)) ||
        (!capturing && (e = cudaEventRecord(b->ev[3], st))))
        return cuda_fail(e, "batched kernel");
    return CF_OK;
}

int batch_run(cf_batch *b, cudaStream_t user, int use_graph, cf_batch_stats *stats)
{
    if (!b)
        return fail(CF_EINVAL, "batch is NULL");
    if (b->jobs.empty())
        return fail(CF_EINVAL, "the batch has no jobs");
    cudaError_t e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)))
        return cuda_fail(e, "cudaGetDevice");
    if (b->dev >= 0 && b->dev != dev)
        return fail(CF_EINVAL, "a batch runs on the device that was current at its first run");
    if (b->dev < 0) {
        b->dev = dev;
        if ((e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev)))
            return cuda_fail(e, "device attribute");
        if ((e = cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking)))
            return cuda_fail(e, "batch stream");
        for (auto &ev : b->ev)
            if ((e = cudaEventCreate(&ev)))
                return cuda_fail(e, "batch events");
    }
    const cudaStream_t st = user ? user : b->own;
    int planned = 0, rc;
    std::vector<std::array<double, 6>> box;
    if ((rc = batch_bboxes(b, st, box)))
        return rc;
    bool same = b->planned;
    for (size_t k = 0; same && k < b->jobs.size(); ++k)
        for (int a = 0; a < 3 && same; ++a)
            same = b->jobs[k].cfg.periodic ||
                   (b->jobs[k].lo[a] == box[k][a] && b->jobs[k].hi[a] == box[k][3 + a]);
    if (!same) {
        if ((rc = batch_plan(b, st, box)))
            return rc;
        planned = 1;
    }
    if (use_graph) {
        if (!b->gexec) {
            // capture on the batch's own stream (the legacy stream cannot capture)
            if ((e = cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal)))
                return cuda_fail(e, "cudaStreamBeginCapture");
            rc = batch_issue(b, b->own, true);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(b->own, &g);
            if (rc) {
                if (g)
                    cudaGraphDestroy(g);
                return rc;
            }
            if (e)
                return cuda_fail(e, "cudaStreamEndCapture");
            b->graph = g;
            if ((e = cudaGraphInstantiate(&b->gexec, g, 0)))
                return cuda_fail(e, "cudaGraphInstantiate");
        }
        // the graph run is timed from outside the graph
        if ((e = cudaEventRecord(b->ev[0], st)) || (e = cudaGraphLaunch(b->gexec, st)) ||
            (e = cudaEventRecord(b->ev[3], st)))
            return cuda_fail(e, "cudaGraphLaunch");
    } else if ((rc = batch_issue(b, st, false))) {
        return rc;
    }
    if ((e = cudaStreamSynchronize(st)))
        return cuda_fail(e, "batch synchronize");
    float kms = -1.f, tms = 0.f;
    if (!use_graph && cudaEventElapsedTime(&kms, b->ev[1], b->ev[2]) != cudaSuccess)
        kms = -1.f;  // the batched kernel alone is timed only outside a graph
    cudaEventElapsedTime(&tms, b->ev[0], b->ev[3]);
    cudaGetLastError();
    uint64_t pairs = 0;
    for (size_t k = 0; k < b->jobs.size(); ++k) {
        BatchJob &j = b->jobs[k];
        const unsigned long long *o = b->h_out + j.out_off;
        unsigned err = 0, kept = 0;
        std::memcpy(&err, o + j.nslots + 4, 4);
        std::memcpy(&kept, reinterpret_cast<const unsigned *>(o + j.nslots + 4) + 2, 4);
        if (err & cf::ERR_COORD)
            return fail(CF_EINVAL, "batch job " + std::to_string(k) +
                                       ": coordinate outside [0, boxsize) or non-finite");
        if (err & cf::ERR_TIMEOUT)
            return fail(CF_ETIMEOUT, "batch job " + std::to_string(k) + ": a bounded device wait gave up");
        if (err)
            return fail(CF_EDEVICE, "batch job " + std::to_string(k) + ": internal inconsistency");
        cf_result *res = j.q.res;
        const uint64_t mult = j.q.autocorr ? 2u : 1u;
        for (int s = 0; s < j.nslots; ++s) {
            res->npairs[s] = o[s] * mult;
            pairs += res->npairs[s];
        }
        if (res->wsum)
            std::memset(res->wsum, 0, sizeof(double) * j.nslots);
        if (res->ravg)
            std::memset(res->ravg, 0, sizeof(double) * j.nslots);
        res->n_cellpairs = kept;
        res->n_evaluated = 0;
        res->n_rechecked = o[j.nslots + 2];
        res->n_band_violations = 0;
        res->kernel_ms = kms;
        res->total_ms = tms;
        res->n_kernels = j.n_kernels;
        res->refine_used[0] = j.g.reach_x;
        res->refine_used[1] = j.g.reach_y;
        res->refine_used[2] = j.g.reach_z;
        res->chunk_used = j.chunk;
        res->pp_used = j.pp;
        res->tuned = j.tuned;
        res->table_linear = j.P.lut_lin;
    }
    if (stats) {
        stats->n_jobs = b->jobs.size();
        stats->n_kernels = b->n_kernels;
        stats->pairs = pairs;
        stats->used_graph = use_graph ? 1 : 0;
        stats->planned = planned;
        stats->blocks = b->blocks;
        stats->kernel_ms = kms;
        stats->total_ms = tms;
    }
    return CF_OK;
}

}  // namespace

extern "C" {

int cf_batch_create(cf_batch **out)
{
    if (!out)
        return fail(CF_EINVAL, "out is NULL");
    *out = new (std::nothrow) cf_batch();
    return *out ? CF_OK : fail(CF_ENOMEM, "out of host memory");
}

int cf_batch_add_xi(cf_batch *b, int autocorr, const cf_catalog *d1, const cf_catalog *d2,
                    const double *edges, int nedges, const cf_config *cfg, cf_result *res)
{
    if (!edges || nedges < 2)
        return fail(CF_EINVAL, "need at least 2 bin edges");
    Request q;
    q.kind = 0;
    q.autocorr = autocorr ? 1 : 0;
    q.d1 = d1;
    q.d2 = d2;
    q.edges.assign(edges, edges + nedges);
    q.pimax = 0.0;
    q.npibins = 0;
    q.cfg = cfg;
    q.res = res;
    return batch_add(b, q);
}

int cf_batch_add_rp_pi(cf_batch *b, int autocorr, const cf_catalog *d1, const cf_catalog *d2,
                       const double *rp_edges, int n_rp_edges, double pimax, int npibins,
                       const cf_config *cfg, cf_result *res)
{
    if (!rp_edges || n_rp_edges < 2)
        return fail(CF_EINVAL, "need at least 2 rp bin edges");
    Request q;
    q.kind = 1;
    q.autocorr = autocorr ? 1 : 0;
    q.d1 = d1;
    q.d2 = d2;
    q.edges.assign(rp_edges, rp_edges + n_rp_edges);
    q.pimax = pimax;
    q.npibins = npibins;
    q.cfg = cfg;
    q.res = res;
    return batch_add(b, q);
}

int cf_batch_run(cf_batch *b, void *stream, int use_graph, cf_batch_stats *stats)
{
    return batch_run(b, (cudaStream_t)stream, use_graph, stats);
}

int cf_batch_destroy(cf_batch *b)
{
    if (!b)
        return CF_OK;
    batch_free_plan(b);
    if (b->own)
        cudaStreamDestroy(b->own);
    for (auto &ev : b->ev)
        if (ev)
            cudaEventDestroy(ev);
    cudaGetLastError();
    delete b;
    return CF_OK;
}

}  // extern "C"
