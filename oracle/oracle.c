/*
 * Brute-force CPU oracle for cell-list pair counting (Sinha & Garrison,
 * "Corrfunc: blazing fast correlation functions with AVX512F SIMD
 * intrinsics", arXiv:1911.08275).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code with the CUDA implementation.
 *
 * What it computes is the plain definition of a pair-separation histogram,
 * i.e. the naive double loop of Sec. 1.1 (Code 1), with the separations of
 * Sec. 1.1 (Eq. "separations"):
 *   xi:       r^2  = dx^2 + dy^2 + dz^2,   counted iff  Rmin^2 <= r^2 < Rmax^2
 *   rp-pi:    rp^2 = dx^2 + dy^2, pi = |dz|, counted iff
 *             Rmin^2 <= rp^2 < Rmax^2  and  pi < pimax
 * Bins are half-open [e_k, e_{k+1}) and are tested on squared separations
 * (Sec. 2.2, Code 3 / Code 4: the kernels never take a square root to bin).
 *
 * Canonical IEEE-754 binary64 evaluation (round to nearest, no FMA
 * contraction: compile with -ffp-contract=off), in this order:
 *   dx = x_j - x_i; periodic: if dx > L/2 then dx -= L, else if dx < -L/2
 *   then dx += L (minimum image; the paper only says "periodic box");
 *   same for dy, dz;
 *   rp2 = dx*dx + dy*dy;   r2 = rp2 + dz*dz;   E2_k = e_k * e_k;
 *   pi bin edges P_m = (pimax * m) / npibins for m < npibins, P_npibins = pimax.
 *
 * Auto-correlation counts ordered pairs i != j.  Each unordered pair is
 * visited once and counted twice, which is the paper's "double the total
 * number of pairs found at the end" (Sec. 2.1, "Reducing the number of cell
 * pairs"); fl(a - b) = -fl(b - a) and the wrap is sign-symmetric, so r2(i,j)
 * equals r2(j,i) bit for bit.  Cross-correlation counts every (i, j).
 *
 * Weights (the weight_func of Code 1 is fixed to the product w_i * w_j):
 *   wsum_k = sum over counted pairs of w_i * w_j;
 *   rsum_k = sum over counted pairs of r * (w_i * w_j, or 1 if unweighted),
 *            r = sqrt(r2) for xi and sqrt(rp2) for rp-pi (correctly rounded).
 * Both sums use Neumaier compensated summation in fixed-size blocks that are
 * combined in block order, so the result does not depend on thread timing.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

typedef struct {
    double sum;
    double comp;
} nsum;

static void nsum_add(nsum *a, double x)
{
    double t = a->sum + x;
    if (fabs(a->sum) >= fabs(x))
        a->comp += (a->sum - t) + x;
    else
        a->comp += (x - t) + a->sum;
    a->sum = t;
}

static double nsum_value(const nsum *a) { return a->sum + a->comp; }

/* One separation component x_j - x_i, with the minimum-image wrap:
 * if d > L/2 then d - L, else if d < -L/2 then d + L, else d.
 * Written as d + s*L with s in {-1, 0, +1}: s*L is exactly -L, 0 or +L, so
 * the result is the same IEEE sum as the branchy form (d + 0 only turns a
 * -0 into +0, which squares identically), and the compiler emits no
 * data-dependent branch. */
static double component(double xi, double xj, int periodic, double L)
{
    const double d = xj - xi;
    if (!periodic)
        return d;
    const int s = (d < -0.5 * L) - (d > 0.5 * L);
    return d + (double)s * L;
}

/* Bin of a squared separation: k with E2[k] <= s < E2[k+1], else -1. */
static int bin_of(double s, const double *E2, int nbins)
{
    if (!(E2[0] <= s && s < E2[nbins]))
        return -1; /* outside [Rmin^2, Rmax^2): no bin can match */
    for (int k = 0; k < nbins; k++)
        if (E2[k] <= s && s < E2[k + 1])
            return k;
    return -1;
}

/* pi bin: m with P[m] <= pi < P[m+1], else -1. */
static int pibin_of(double pi, const double *P, int npibins)
{
    for (int m = 0; m < npibins; m++)
        if (P[m] <= pi && pi < P[m + 1])
            return m;
    return -1;
}

typedef struct {
    int64_t n;
    const double *x, *y, *z, *w;
} cat;

typedef struct {
    int kind; /* 0 = xi, 1 = rp-pi */
    int autocorr, periodic;
    double box[3];
    int nbins;       /* radial (xi) or rp bins */
    const double *E2; /* nbins + 1 squared edges */
    int npibins;     /* rp-pi only */
    const double *P; /* npibins + 1 pi edges */
    int weighted, want_r;
} job;

/* Accumulate the pairs of primary rows [i0, i1) into one block's histograms. */
static void count_rows(const job *jb, const cat *a, const cat *b, int64_t i0, int64_t i1,
                       uint64_t *restrict cnt, nsum *restrict ws, nsum *restrict rs)
{
    const double *restrict bx = b->x, *restrict by = b->y, *restrict bz = b->z;
    const int64_t nb = b->n;
    const int periodic = jb->periodic;
    const double Lx = jb->box[0], Ly = jb->box[1], Lz = jb->box[2];
    const uint64_t mult = jb->autocorr ? 2u : 1u;
    for (int64_t i = i0; i < i1; i++) {
        const double xi = a->x[i], yi = a->y[i], zi = a->z[i];
        const int64_t j0 = jb->autocorr ? i + 1 : 0;
        for (int64_t j = j0; j < nb; j++) {
            const double dx = component(xi, bx[j], periodic, Lx);
            const double dy = component(yi, by[j], periodic, Ly);
            const double dz = component(zi, bz[j], periodic, Lz);
            const double rp2 = dx * dx + dy * dy;
            int slot;
            double s;
            if (jb->kind == 0) {
                const double r2 = rp2 + dz * dz;
                const int k = bin_of(r2, jb->E2, jb->nbins);
                if (k < 0)
                    continue;
                slot = k;
                s = r2;
            } else {
                const int k = bin_of(rp2, jb->E2, jb->nbins);
                if (k < 0)
                    continue;
                const int m = pibin_of(fabs(dz), jb->P, jb->npibins);
                if (m < 0)
                    continue;
                slot = k * jb->npibins + m;
                s = rp2;
            }
            cnt[slot] += mult;
            double pw = 1.0;
            if (jb->weighted) {
                pw = a->w[i] * b->w[j];
                nsum_add(&ws[slot], pw);
                if (jb->autocorr)
                    nsum_add(&ws[slot], pw);
            }
            if (jb->want_r) {
                const double rv = sqrt(s) * pw;
                nsum_add(&rs[slot], rv);
                if (jb->autocorr)
                    nsum_add(&rs[slot], rv);
            }
        }
    }
}

static int run(const job *jb, const cat *a, const cat *b, uint64_t *npairs, double *wsum,
               double *rsum)
{
    const int nslots = jb->kind == 0 ? jb->nbins : jb->nbins * jb->npibins;
    /* Fixed row blocks, combined in block order: results independent of threads. */
    const int64_t nblk = a->n < 1024 ? (a->n > 0 ? a->n : 1) : 1024;
    uint64_t *cnt = calloc((size_t)nblk * nslots, sizeof(uint64_t));
    nsum *ws = calloc((size_t)nblk * nslots, sizeof(nsum));
    nsum *rs = calloc((size_t)nblk * nslots, sizeof(nsum));
    if (!cnt || !ws || !rs) {
        free(cnt);
        free(ws);
        free(rs);
        return ORACLE_ENOMEM;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t blk = 0; blk < nblk; blk++) {
        /* Auto-correlation rows shrink with i: interleave rows across blocks. */
        if (jb->autocorr) {
            for (int64_t i = blk; i < a->n; i += nblk)
                count_rows(jb, a, b, i, i + 1, cnt + blk * nslots, ws + blk * nslots,
                           rs + blk * nslots);
        } else {
            int64_t i0 = a->n * blk / nblk, i1 = a->n * (blk + 1) / nblk;
            count_rows(jb, a, b, i0, i1, cnt + blk * nslots, ws + blk * nslots, rs + blk * nslots);
        }
    }
    for (int s = 0; s < nslots; s++) {
        uint64_t c = 0;
        nsum W = {0.0, 0.0}, R = {0.0, 0.0};
        for (int64_t blk = 0; blk < nblk; blk++) {
            c += cnt[blk * nslots + s];
            nsum_add(&W, nsum_value(&ws[blk * nslots + s]));
            nsum_add(&R, nsum_value(&rs[blk * nslots + s]));
        }
        npairs[s] = c;
        if (wsum)
            wsum[s] = nsum_value(&W);
        if (rsum)
            rsum[s] = nsum_value(&R);
    }
    free(cnt);
    free(ws);
    free(rs);
    return ORACLE_OK;
}

static int check_common(int autocorr, const cat *a, const cat *b, int periodic,
                        const double *box, const double *edges, int nedges)
{
    if (!a || a->n < 0 || !edges || nedges < 2)
        return ORACLE_EINVAL;
    if (!autocorr && (!b || b->n < 0))
        return ORACLE_EINVAL;
    if (edges[0] < 0.0)
        return ORACLE_EINVAL;
    for (int k = 0; k + 1 < nedges; k++)
        if (!(edges[k] < edges[k + 1]))
            return ORACLE_EINVAL;
    if (periodic && !box)
        return ORACLE_EINVAL;
    return ORACLE_OK;
}

/*
 * DD(r): histogram of r^2 against squared edges (Sec. 1.1 Code 1 and
 * Eq. "separations"; Code 4 for squared-edge binning).
 *   autocorr: 1 -> pairs within catalogue 1 (x2.. ignored), 0 -> 1 x 2.
 *   w1, w2: NULL for unweighted; wsum may be NULL.  rsum may be NULL.
 *   npairs[nedges-1], wsum[nedges-1], rsum[nedges-1] are caller-owned.
 */
int oracle_xi(int autocorr, int64_t n1, const double *x1, const double *y1, const double *z1,
              const double *w1, int64_t n2, const double *x2, const double *y2,
              const double *z2, const double *w2, int periodic, const double *box,
              const double *edges, int nedges, uint64_t *npairs, double *wsum, double *rsum)
{
    cat a = {n1, x1, y1, z1, w1};
    cat b = autocorr ? a : (cat){n2, x2, y2, z2, w2};
    int st = check_common(autocorr, &a, &b, periodic, box, edges, nedges);
    if (st)
        return st;
    int weighted = w1 != NULL;
    if (weighted && !autocorr && !w2)
        return ORACLE_EINVAL;
    double *E2 = malloc(sizeof(double) * nedges);
    if (!E2)
        return ORACLE_ENOMEM;
    for (int k = 0; k < nedges; k++)
        E2[k] = edges[k] * edges[k];
    job jb = {0, autocorr, periodic, {0, 0, 0}, nedges - 1, E2, 0, NULL, weighted, rsum != NULL};
    if (periodic)
        memcpy(jb.box, box, sizeof(jb.box));
    st = run(&jb, &a, &b, npairs, weighted ? wsum : NULL, rsum);
    if (!weighted && wsum)
        for (int k = 0; k < nedges - 1; k++)
            wsum[k] = 0.0;
    free(E2);
    return st;
}

/*
 * DD(rp, pi): 2-D histogram, rp-major: npairs[k * npibins + m] for rp bin k
 * ([e_k, e_{k+1}) on rp^2) and pi bin m ([P_m, P_{m+1}) on |dz|), counted iff
 * pi < pimax (Eq. "separations"; line of sight = z).
 */
int oracle_rppi(int autocorr, int64_t n1, const double *x1, const double *y1, const double *z1,
                const double *w1, int64_t n2, const double *x2, const double *y2,
                const double *z2, const double *w2, int periodic, const double *box,
                const double *rp_edges, int n_rp_edges, double pimax, int npibins,
                uint64_t *npairs, double *wsum, double *rsum)
{
    cat a = {n1, x1, y1, z1, w1};
    cat b = autocorr ? a : (cat){n2, x2, y2, z2, w2};
    int st = check_common(autocorr, &a, &b, periodic, box, rp_edges, n_rp_edges);
    if (st)
        return st;
    if (!(pimax > 0.0) || npibins < 1)
        return ORACLE_EINVAL;
    int weighted = w1 != NULL;
    if (weighted && !autocorr && !w2)
        return ORACLE_EINVAL;
    double *E2 = malloc(sizeof(double) * n_rp_edges);
    double *P = malloc(sizeof(double) * (npibins + 1));
    if (!E2 || !P) {
        free(E2);
        free(P);
        return ORACLE_ENOMEM;
    }
    for (int k = 0; k < n_rp_edges; k++)
        E2[k] = rp_edges[k] * rp_edges[k];
    for (int m = 0; m < npibins; m++)
        P[m] = (pimax * (double)m) / (double)npibins;
    P[npibins] = pimax;
    job jb = {1, autocorr, periodic, {0, 0, 0}, n_rp_edges - 1, E2, npibins, P, weighted,
              rsum != NULL};
    if (periodic)
        memcpy(jb.box, box, sizeof(jb.box));
    const int nslots = (n_rp_edges - 1) * npibins;
    st = run(&jb, &a, &b, npairs, weighted ? wsum : NULL, rsum);
    if (!weighted && wsum)
        for (int k = 0; k < nslots; k++)
            wsum[k] = 0.0;
    free(E2);
    free(P);
    return st;
}

/* Threads the oracle uses (for reporting the CPU baseline's core count). */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
