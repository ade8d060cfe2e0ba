/*
 * Plain gridded CPU pair counter for DD(r): the CPU baseline of the benchmark.
 *
 * BASELINE AND TEST INFRASTRUCTURE ONLY.  Like the brute-force oracle in this
 * directory, nothing in the product path may call, link or load it: only the
 * tests and the CPU legs of the benchmark use it.  It shares no code with the
 * CUDA implementation.  The tests pin its counts to the brute-force oracle bit
 * for bit.
 *
 * It is the cell-list method of Sinha & Garrison (arXiv:1911.08275) without
 * SIMD:
 *   - Sec. 1.2 / 2.1: points are binned into cells of side at least
 *     Rmax / refine along each axis (refine defaults to the paper's (2, 2, 1),
 *     Sec. 3.1), so every pair closer than Rmax lies in cells at most refine
 *     apart; the points of a cell are stored contiguously, sorted along z;
 *   - Sec. 2.1: an auto-correlation visits each unordered pair of cells once
 *     (half of the neighbour offsets, the cell with itself for j > i) and
 *     doubles the counts;
 *   - Sec. 2.2 (Code 2): along the sorted z axis, secondaries that lie Rmax or
 *     more below the primary are skipped (late entry) and the scan stops at the
 *     first one Rmax or more above it (early exit);
 *   - Sec. 1.1 (Code 1), Code 3 / Code 4: every remaining pair's squared
 *     separation is computed and binned against squared edges.
 *
 * The arithmetic is the canonical binary64 one of the oracle (round to
 * nearest, no FMA contraction: compile with -ffp-contract=off):
 *   dx = x_j - x_i, plus the periodic image shift S_x in {-L, 0, +L} of the
 *   cell pair (for a pair closer than L/2 this is the oracle's minimum-image
 *   wrap, bit for bit); rp2 = dx*dx + dy*dy; r2 = rp2 + dz*dz;
 *   bin k iff e_k^2 <= r2 < e_{k+1}^2.
 * The z skips only drop pairs with |dz| >= Rmax, whose r2 >= Rmax^2 (rounding
 * is monotone), so the counts equal the oracle's exactly.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GRID_OK 0
#define GRID_EINVAL (-1)
#define GRID_ENOMEM (-2)

typedef struct {
    int64_t n;
    double *x, *y, *z;  /* points in cell order (cells sorted by z inside) */
    int64_t *start;     /* ncells + 1 */
} grid;

typedef struct {
    int n[3];            /* cells per axis */
    double origin[3], inv_w[3];
    int64_t ncells;
} geom;

static int cell_axis(double v, const geom *g, int a)
{
    double t = floor((v - g->origin[a]) * g->inv_w[a]);
    if (t < 0.0)
        t = 0.0;
    if (t > (double)(g->n[a] - 1))
        t = (double)(g->n[a] - 1);
    return (int)t;
}

static int64_t cell_of(double x, double y, double z, const geom *g)
{
    const int cx = cell_axis(x, g, 0), cy = cell_axis(y, g, 1), cz = cell_axis(z, g, 2);
    return ((int64_t)cx * g->n[1] + cy) * g->n[2] + cz;
}

typedef struct {
    double z;
    int64_t i;
} zkey;

static int cmp_zkey(const void *a, const void *b)
{
    const zkey *p = (const zkey *)a, *q = (const zkey *)b;
    if (p->z < q->z)
        return -1;
    if (p->z > q->z)
        return 1;
    return (p->i > q->i) - (p->i < q->i);
}

/* Counting sort of the points by cell, then each cell sorted by z. */
static int build_grid(int64_t n, const double *x, const double *y, const double *z, const geom *g,
                      grid *out)
{
    out->n = n;
    out->x = malloc(sizeof(double) * (n > 0 ? n : 1));
    out->y = malloc(sizeof(double) * (n > 0 ? n : 1));
    out->z = malloc(sizeof(double) * (n > 0 ? n : 1));
    out->start = calloc((size_t)g->ncells + 1, sizeof(int64_t));
    int64_t *cell = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    int64_t *fill = malloc(sizeof(int64_t) * ((size_t)g->ncells + 1));
    zkey *keys = malloc(sizeof(zkey) * (n > 0 ? n : 1));
    if (!out->x || !out->y || !out->z || !out->start || !cell || !fill || !keys) {
        free(cell);
        free(fill);
        free(keys);
        return GRID_ENOMEM;
    }
    for (int64_t i = 0; i < n; i++) {
        cell[i] = cell_of(x[i], y[i], z[i], g);
        out->start[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < g->ncells; c++)
        out->start[c + 1] += out->start[c];
    memcpy(fill, out->start, sizeof(int64_t) * (size_t)g->ncells);
    for (int64_t i = 0; i < n; i++)
        keys[fill[cell[i]]++] = (zkey){z[i], i};
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t c = 0; c < g->ncells; c++) {
        const int64_t a = out->start[c], b = out->start[c + 1];
        if (b - a > 1)
            qsort(keys + a, (size_t)(b - a), sizeof(zkey), cmp_zkey);
        for (int64_t k = a; k < b; k++) {
            const int64_t i = keys[k].i;
            out->x[k] = x[i];
            out->y[k] = y[i];
            out->z[k] = z[i];
        }
    }
    free(cell);
    free(fill);
    free(keys);
    return GRID_OK;
}

static void free_grid(grid *g)
{
    free(g->x);
    free(g->y);
    free(g->z);
    free(g->start);
}

/* Bin of a squared separation: k with E2[k] <= s < E2[k+1], else -1. */
static int bin_of(double s, const double *E2, int nbins)
{
    if (!(E2[0] <= s && s < E2[nbins]))
        return -1;
    int lo = 0, hi = nbins; /* E2[lo] <= s < E2[hi] */
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (E2[mid] <= s)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

static int floor_div(int a, int n) { return a >= 0 ? a / n : -((-a + n - 1) / n); }

/*
 * DD(r) by cell lists.
 *   autocorr 1: ordered pairs i != j of catalogue 1 (catalogue 2 ignored);
 *            0: every (i in 1, j in 2).
 *   periodic 1: box[3] per axis, coordinates in [0, box) and Rmax < box/2;
 *            0: the grid covers the bounding box of both catalogues.
 *   refine   cells per Rmax along x, y, z (NULL: the paper's (2, 2, 1)).
 *   npairs   nedges - 1 counts (ordered pairs), caller-owned.
 */
int gridded_xi(int autocorr, int64_t n1, const double *x1, const double *y1, const double *z1,
               int64_t n2, const double *x2, const double *y2, const double *z2, int periodic,
               const double *box, const double *edges, int nedges, const int *refine,
               uint64_t *npairs)
{
    if (n1 < 0 || (!autocorr && n2 < 0) || !edges || nedges < 2 || !npairs || (periodic && !box))
        return GRID_EINVAL;
    for (int k = 0; k + 1 < nedges; k++)
        if (!(edges[k] < edges[k + 1]) || edges[0] < 0.0)
            return GRID_EINVAL;
    const int nb = nedges - 1;
    const double R = edges[nb];
    const int r[3] = {refine ? refine[0] : 2, refine ? refine[1] : 2, refine ? refine[2] : 1};
    for (int a = 0; a < 3; a++)
        if (r[a] < 1 || r[a] > 16)
            return GRID_EINVAL;
    if (autocorr) {
        n2 = n1;
        x2 = x1;
        y2 = y1;
        z2 = z1;
    }
    memset(npairs, 0, sizeof(uint64_t) * nb);
    if (n1 == 0 || n2 == 0)
        return GRID_OK;

    /* geometry: cells of side >= Rmax (1 + 1e-9) / refine, so that two points
     * closer than Rmax are at most refine cells apart despite rounding */
    geom g;
    double ext[3];
    for (int a = 0; a < 3; a++) {
        if (periodic) {
            if (!(R < 0.5 * box[a]))
                return GRID_EINVAL;
            g.origin[a] = 0.0;
            ext[a] = box[a];
        } else {
            const double *v1 = a == 0 ? x1 : (a == 1 ? y1 : z1);
            const double *v2 = a == 0 ? x2 : (a == 1 ? y2 : z2);
            double lo = v1[0], hi = v1[0];
            for (int64_t i = 0; i < n1; i++) {
                lo = fmin(lo, v1[i]);
                hi = fmax(hi, v1[i]);
            }
            for (int64_t i = 0; i < n2; i++) {
                lo = fmin(lo, v2[i]);
                hi = fmax(hi, v2[i]);
            }
            g.origin[a] = lo;
            ext[a] = fmax(hi - lo, 1e-300);
        }
        double per = floor(ext[a] / (R * (1.0 + 1e-9)));
        if (per < 1.0)
            per = 1.0;
        if (per > 1024.0)
            per = 1024.0;
        g.n[a] = (int)per * r[a];
    }
    /* at most 2^24 cells: coarsen the finest axis (wider cells stay correct) */
    while ((int64_t)g.n[0] * g.n[1] * g.n[2] > ((int64_t)1 << 24)) {
        int a = 0;
        for (int d = 1; d < 3; d++)
            if (g.n[d] / r[d] > g.n[a] / r[a])
                a = d;
        g.n[a] = (g.n[a] / r[a] / 2 > 1 ? g.n[a] / r[a] / 2 : 1) * r[a];
    }
    for (int a = 0; a < 3; a++)
        g.inv_w[a] = g.n[a] / ext[a];
    g.ncells = (int64_t)g.n[0] * g.n[1] * g.n[2];

    grid A, B;
    memset(&A, 0, sizeof(A));
    memset(&B, 0, sizeof(B));
    int st = build_grid(n1, x1, y1, z1, &g, &A);
    if (st == GRID_OK && !autocorr)
        st = build_grid(n2, x2, y2, z2, &g, &B);
    if (st != GRID_OK) {
        free_grid(&A);
        free_grid(&B);
        return st;
    }
    const grid *pb = autocorr ? &A : &B;

    double *E2 = malloc(sizeof(double) * nedges);
    if (!E2) {
        free_grid(&A);
        free_grid(&B);
        return GRID_ENOMEM;
    }
    for (int k = 0; k < nedges; k++)
        E2[k] = edges[k] * edges[k];

    /* neighbour offsets: all of [-r, r]^3, or half of them for auto (Sec. 2.1) */
    const int sx = 2 * r[0] + 1, sy = 2 * r[1] + 1, sz = 2 * r[2] + 1;
    int (*off)[3] = malloc(sizeof(int[3]) * (size_t)sx * sy * sz);
    int noff = 0;
    if (!off) {
        free(E2);
        free_grid(&A);
        free_grid(&B);
        return GRID_ENOMEM;
    }
    for (int ox = -r[0]; ox <= r[0]; ox++)
        for (int oy = -r[1]; oy <= r[1]; oy++)
            for (int oz = -r[2]; oz <= r[2]; oz++) {
                if (autocorr && !(ox > 0 || (ox == 0 && (oy > 0 || (oy == 0 && oz >= 0)))))
                    continue;
                off[noff][0] = ox;
                off[noff][1] = oy;
                off[noff][2] = oz;
                noff++;
            }

    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    uint64_t *cnt = calloc((size_t)nthreads * nb, sizeof(uint64_t));
    if (!cnt) {
        free(off);
        free(E2);
        free_grid(&A);
        free_grid(&B);
        return GRID_ENOMEM;
    }

#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        uint64_t *h = cnt + (size_t)tid * nb;
#pragma omp for schedule(dynamic, 16)
        for (int64_t ca = 0; ca < g.ncells; ca++) {
            const int64_t a0 = A.start[ca], a1 = A.start[ca + 1];
            if (a0 == a1)
                continue;
            const int ax = (int)(ca / ((int64_t)g.n[1] * g.n[2]));
            const int ay = (int)((ca / g.n[2]) % g.n[1]);
            const int az = (int)(ca % g.n[2]);
            for (int o = 0; o < noff; o++) {
                int c[3] = {ax + off[o][0], ay + off[o][1], az + off[o][2]};
                double S[3] = {0.0, 0.0, 0.0};
                int outside = 0;
                for (int d = 0; d < 3; d++) {
                    if (periodic) {
                        const int q = floor_div(c[d], g.n[d]);
                        c[d] -= q * g.n[d];
                        /* an image two or more boxes away holds no pair within Rmax < L/2 */
                        if (q < -1 || q > 1)
                            outside = 1;
                        S[d] = (double)q * box[d];
                    } else if (c[d] < 0 || c[d] >= g.n[d]) {
                        outside = 1;
                    }
                }
                if (outside)
                    continue;
                const int64_t cb = ((int64_t)c[0] * g.n[1] + c[1]) * g.n[2] + c[2];
                const int64_t b0 = pb->start[cb], b1 = pb->start[cb + 1];
                if (b0 == b1)
                    continue;
                const int self = autocorr && off[o][0] == 0 && off[o][1] == 0 && off[o][2] == 0;
                int64_t jlo = b0; /* late entry: first j with dz > -Rmax for the current i */
                for (int64_t i = a0; i < a1; i++) {
                    const double xi = A.x[i], yi = A.y[i], zi = A.z[i];
                    int64_t j = self ? i + 1 : jlo;
                    if (!self) {
                        /* z_i grows with i: the late-entry point only moves forward */
                        while (j < b1) {
                            double dz = pb->z[j] - zi;
                            if (S[2] != 0.0)
                                dz = dz + S[2];
                            if (dz > -R)
                                break;
                            j++;
                        }
                        jlo = j;
                    }
                    for (; j < b1; j++) {
                        double dz = pb->z[j] - zi;
                        if (S[2] != 0.0)
                            dz = dz + S[2];
                        if (dz >= R)
                            break; /* early exit: every later j is further in z */
                        double dx = pb->x[j] - xi, dy = pb->y[j] - yi;
                        if (S[0] != 0.0)
                            dx = dx + S[0];
                        if (S[1] != 0.0)
                            dy = dy + S[1];
                        const double rp2 = dx * dx + dy * dy;
                        const double r2 = rp2 + dz * dz;
                        const int k = bin_of(r2, E2, nb);
                        if (k >= 0)
                            h[k]++;
                    }
                }
            }
        }
    }
    const uint64_t mult = autocorr ? 2u : 1u;
    for (int t = 0; t < nthreads; t++)
        for (int k = 0; k < nb; k++)
            npairs[k] += cnt[(size_t)t * nb + k] * mult;
    free(cnt);
    free(off);
    free(E2);
    free_grid(&A);
    free_grid(&B);
    return GRID_OK;
}

/* Threads the counter uses (for reporting the baseline's core count). */
int gridded_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
