/*
 * hdmc_oracle.c -- plain serial reference implementation of the massively
 * parallel hard-disk Monte Carlo sweep (Anderson, Jankowski, Grubb, Engel,
 * Glotzer, "Massively parallel Monte Carlo for many-particle simulations on
 * GPUs", J. Comput. Phys. 2013).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or
 * constant generator with the CUDA library; both sides implement Philox4x32-10
 * independently from its published definition (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11).
 *
 * Everything here is deliberately plain: one cell at a time, in the order of
 * the paper's pseudocode, no blocking, no fusion.  Build with
 *     gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared
 * (-ffp-contract=off matters: the GPU path must agree bit for bit, and gcc on
 * aarch64 would otherwise fuse a*b+c into one rounding).  An optional
 * -fopenmp runs the cells of one checkerboard set in parallel; cells of one
 * set never read each other's data (Sec. 2.1), so the result is identical for
 * any thread count.
 *
 * Two arithmetic modes, fixed at creation:
 *   prec 0 (FP64): positions are binary64 cell-local offsets.
 *   prec 1 (FP32): positions are binary32 cell-local offsets (the paper stores
 *                  single-precision coordinates, Sec. 5); the cell widths used
 *                  inside the sweep are the binary32 roundings of wx, wy.  The
 *                  grid shift alone is evaluated in binary64 (translation,
 *                  ownership test and re-expression, on the binary32 widths)
 *                  and rounded to binary32 once, when it is stored; the grid
 *                  origin accumulates the binary64 shift distance.
 *
 * Readings of the paper taken here (each one is listed in the design notes):
 *  - a cell is the half-open square [0,wx) x [0,wy) in its own frame (Alg. 4
 *    writes 0 < D <= w, Alg. 2 leaves "in cell" unstated);
 *  - containment is tested before overlap (same accepted set, Alg. 2);
 *  - the own-cell overlap candidates are the cell's current (shuffled)
 *    positions other than the moving one (Alg. 2 reads them from global
 *    memory, which would be stale);
 *  - the trial displacement is uniform over a disk of radius d, drawn by
 *    rejection from a symmetric lattice of points in (-1,1)^2;
 *  - the grid is mx x my cells, mx (my) the largest even integer <= Lx/sigma
 *    (Ly/sigma), so that the checkerboard tiles the periodic box (Eq. 1);
 *  - a migrant re-expressed in the new cell's frame that rounds onto the
 *    upper cell edge is clamped to the largest representable value below it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_EOVERFLOW 3
#define ORC_EOVERLAP 4
#define ORC_ENOMEM 6

#define NMAX 4               /* disks per cell when sigma <= w < sqrt(2) sigma (Sec. 3.1, Fig. 3) */
#define EMPTY_SLOT (-1.0e4)  /* exported value of an unused slot (Sec. 3.2 uses (-10,-10)) */

/* Philox counter word 2 carries the stream's domain in bits 28..31. */
#define DOM_SHUFFLE 0u
#define DOM_TRIAL 1u
#define DOM_SWEEP 2u
#define DOM_INIT 3u
#define DOM_SHIFT 4u

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. SC'11): ten rounds of two 32x32->64 products */
/* mixed with the counter and a Weyl-sequence key.                           */
/* ------------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(prod1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)prod1;
        uint32_t y2 = (uint32_t)(prod0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)prod0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* A stream of 32-bit words: block b of the stream is Philox(key, (c0,c1,c2,b)),
 * and its four words are consumed in order. */
typedef struct {
    uint32_t key[2];
    uint32_t c0, c1, c2;
    uint32_t block;
    uint32_t buf[4];
    int pos;
} stream_t;

static void stream_open(stream_t *s, uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2)
{
    s->key[0] = (uint32_t)seed;
    s->key[1] = (uint32_t)(seed >> 32);
    s->c0 = c0; s->c1 = c1; s->c2 = c2;
    s->block = 0;
    s->pos = 4;
}

static uint32_t stream_word(stream_t *s)
{
    if (s->pos == 4) {
        uint32_t ctr[4] = {s->c0, s->c1, s->c2, s->block};
        orc_philox(ctr, s->key, s->buf);
        s->block += 1;
        s->pos = 0;
    }
    return s->buf[s->pos++];
}

/* Uniform integer in [0, range), 1 <= range < 2^32, by Lemire's multiply-high
 * method with exact rejection (Lemire, "Fast random integer generation in an
 * interval", ACM TOMACS 2019): the low half of word*range is rejected when it
 * falls below 2^32 mod range. */
static int lemire_map(uint32_t word, uint32_t range, uint32_t *value)
{
    uint32_t threshold = (uint32_t)(0u - range) % range; /* 2^32 mod range */
    uint64_t m = (uint64_t)word * (uint64_t)range;
    *value = (uint32_t)(m >> 32);
    return (uint32_t)m >= threshold;
}

static uint32_t stream_bounded(stream_t *s, uint32_t range)
{
    uint32_t value;
    while (!lemire_map(stream_word(s), range, &value)) {
    }
    return value;
}

/* Symmetric binary64 variate: k = top 52 bits of (hi:lo), value (2k+1-2^52) 2^-52.
 * The 2^52 values are the odd multiples of 2^-52 in (-1,1), mirror-symmetric
 * about 0, each exactly representable. */
static double sym52(uint32_t hi, uint32_t lo)
{
    uint64_t k = (((uint64_t)hi << 32) | (uint64_t)lo) >> 12;
    int64_t m = (int64_t)(2 * k + 1) - ((int64_t)1 << 52);
    return (double)m * 0x1p-52;
}

/* Uniform binary64 in [0,1) with 53 random bits. */
static double unif53(uint32_t hi, uint32_t lo)
{
    uint64_t k = (((uint64_t)hi << 32) | (uint64_t)lo) >> 11;
    return (double)k * 0x1p-53;
}

/* Exposed for the tests. */
uint32_t orc_stream_bounded(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                            uint32_t range, int64_t count, uint32_t *out)
{
    stream_t s;
    stream_open(&s, seed, c0, c1, c2);
    for (int64_t i = 0; i < count; ++i)
        out[i] = stream_bounded(&s, range);
    return s.block;
}

void orc_stream_words(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                      int64_t count, uint32_t *out)
{
    stream_t s;
    stream_open(&s, seed, c0, c1, c2);
    for (int64_t i = 0; i < count; ++i)
        out[i] = stream_word(&s);
}

/* Lemire acceptance count over every 32-bit word for one range <= 16
 * (exhaustive test of exact uniformity): counts[v] = #words mapping to v. */
void orc_lemire_exhaustive(uint32_t range, uint64_t *counts)
{
    memset(counts, 0, sizeof(uint64_t) * range);
    /* 2^32 words split into 256 chunks (parallel when built with OpenMP). */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int chunk = 0; chunk < 256; ++chunk) {
        uint64_t local[16] = {0};
        uint32_t w0 = (uint32_t)chunk << 24;
        for (uint32_t k = 0; k < (1u << 24); ++k) {
            uint32_t v;
            if (lemire_map(w0 + k, range, &v)) local[v & 15] += 1;
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        for (uint32_t v = 0; v < range && v < 16; ++v) counts[v] += local[v];
    }
}

double orc_sym52(uint32_t hi, uint32_t lo) { return sym52(hi, lo); }

/* ------------------------------------------------------------------------ */
/* System state                                                              */
/* ------------------------------------------------------------------------ */
typedef struct oracle {
    int64_t N;
    double Lx, Ly, sigma, d;
    int nsel;
    uint64_t seed;
    int prec;
    int mx, my;
    double wx, wy;          /* cell widths, binary64 */
    float wxf, wyf;         /* binary32 cell widths used by the FP32 mode */
    int64_t C;              /* mx*my */
    double *X, *Y;          /* FP64 mode: slot (c,j) at index 4c+j, canonical c = cy*mx+cx */
    float *Xf, *Yf;         /* FP32 mode */
    uint8_t *n;             /* disks per cell */
    double Ox, Oy;          /* accumulated grid origin (Alg. 1, shift_cells) */
    uint64_t sweep;         /* index of the next sweep */
    uint64_t shifts;        /* explicit shifts done so far */
    uint64_t cnt[4];        /* trials, accepted, rejected (left cell), rejected (overlap) */
    /* balance-control switches (Sec. 2.4): 1 = step performed (default) */
    int shuffle_particles, shuffle_sets;
    /* negative control of Sec. 2.4 item 1 (both modes, serial order): 1 = a
     * trial position outside the cell moves the disk into the neighbouring cell */
    int allow_leave;
    /* spatial decomposition with inactive bands (Sec. 6): 0 = none; else the
     * rows form nstrips strips and the first row of each strip makes no
     * trial moves (band[cy] = 1) */
    int nstrips;
    uint8_t *band;
} oracle_t;

static double prev_double(double w) { return nextafter(w, 0.0); }
static float prev_float(float w) { return nextafterf(w, 0.0f); }

/* binary32 overlap predicate: dx^2 + dy^2 < sigma^2 evaluated as
 * fma(dx, dx, fma(dy, dy, -sigma^2)) < 0 (two roundings).  The binary64
 * predicate is dx*dx + dy*dy < sigma^2 with three roundings. */
static int overlap32(float dx, float dy, float sig2)
{
    return fmaf(dx, dx, fmaf(dy, dy, -sig2)) < 0.0f;
}

/* Grid rules (both give an even m, which the checkerboard of Eq. 1 needs on a
 * periodic box, and sigma <= w < sqrt(2) sigma, so a cell holds at most four
 * centres, Fig. 3):
 *   0: m = largest even integer <= L/sigma (cells just wider than sigma);
 *   1: the paper's rule of Sec. 3.1, m = floor(L/(sqrt(2) sigma)) rounded up:
 *      the smallest even m > L/(sqrt(2) sigma), the widest cells that still
 *      hold at most four centres. */
#define CELLS_SQRT2 1
static int grid_size_rule(double L, double sigma, int rule)
{
    double q = floor(L / sigma);
    if (q > 2.0e9) return -1;
    int m = (int)q;
    m -= m & 1;
    if (rule == CELLS_SQRT2) {
        double r = floor(L / (sqrt(2.0) * sigma)) + 1.0;
        int k = (int)r;
        k += k & 1;
        if (k > m) return -1;   /* w would fall below sigma */
        m = k;
    }
    return m;
}

static int grid_size(double L, double sigma) { return grid_size_rule(L, sigma, 0); }

int orc_grid_rule(double Lx, double Ly, double sigma, int rule, int32_t *mx, int32_t *my, double *wx, double *wy)
{
    if (!(sigma > 0) || !(Lx > 0) || !(Ly > 0) || rule < 0 || rule > 1) return ORC_EINVAL;
    int a = grid_size_rule(Lx, sigma, rule), b = grid_size_rule(Ly, sigma, rule);
    if (a < 4 || b < 4) return ORC_EINVAL;
    *mx = a; *my = b;
    *wx = Lx / a; *wy = Ly / b;
    /* n <= 4 needs w < sqrt(2) sigma (Fig. 3): compare w^2 < 2 sigma^2 */
    if (!((*wx) * (*wx) < 2.0 * sigma * sigma) || !((*wy) * (*wy) < 2.0 * sigma * sigma))
        return ORC_EINVAL;
    return ORC_OK;
}

int orc_grid(double Lx, double Ly, double sigma, int32_t *mx, int32_t *my, double *wx, double *wy)
{
    return orc_grid_rule(Lx, Ly, sigma, 0, mx, my, wx, wy);
}

static int is_set(const oracle_t *o, int64_t c, int j) { return j < o->n[c]; }

static void slot_get(const oracle_t *o, int64_t c, int j, double *x, double *y)
{
    if (o->prec == 0) { *x = o->X[4 * c + j]; *y = o->Y[4 * c + j]; }
    else { *x = (double)o->Xf[4 * c + j]; *y = (double)o->Yf[4 * c + j]; }
}

void orc_destroy(oracle_t *o)
{
    if (!o) return;
    free(o->X); free(o->Y); free(o->Xf); free(o->Yf); free(o->n); free(o->band);
    free(o);
}

static oracle_t *alloc_state(int64_t N, double Lx, double Ly, double sigma, double d,
                             int nsel, uint64_t seed, int prec, int *err)
{
    int32_t mx, my;
    double wx, wy;
    *err = ORC_EINVAL;
    /* prec: arithmetic mode (bits 0-7), optionally + 256 * grid rule */
    int rule = prec >> 8;
    prec &= 0xFF;
    if (N < 1 || nsel < 1 || nsel > 255 || (prec != 0 && prec != 1)) return NULL;
    if (orc_grid_rule(Lx, Ly, sigma, rule, &mx, &my, &wx, &wy) != ORC_OK) return NULL;
    if (!(d > 0) || !(d < 0.5 * wx) || !(d < 0.5 * wy)) return NULL;
    if ((int64_t)mx * my * NMAX < N) return NULL;
    oracle_t *o = (oracle_t *)calloc(1, sizeof(oracle_t));
    *err = ORC_ENOMEM;
    if (!o) return NULL;
    o->N = N; o->Lx = Lx; o->Ly = Ly; o->sigma = sigma; o->d = d;
    o->nsel = nsel; o->seed = seed; o->prec = prec;
    o->mx = mx; o->my = my; o->wx = wx; o->wy = wy;
    o->wxf = (float)wx; o->wyf = (float)wy;
    o->C = (int64_t)mx * my;
    o->shuffle_particles = 1; o->shuffle_sets = 1;
    o->n = (uint8_t *)calloc((size_t)o->C, 1);
    if (prec == 0) {
        o->X = (double *)malloc(sizeof(double) * 4 * (size_t)o->C);
        o->Y = (double *)malloc(sizeof(double) * 4 * (size_t)o->C);
        if (!o->X || !o->Y || !o->n) { orc_destroy(o); return NULL; }
    } else {
        o->Xf = (float *)malloc(sizeof(float) * 4 * (size_t)o->C);
        o->Yf = (float *)malloc(sizeof(float) * 4 * (size_t)o->C);
        if (!o->Xf || !o->Yf || !o->n) { orc_destroy(o); return NULL; }
    }
    *err = ORC_OK;
    return o;
}

/* Bin one global position (x in [0,Lx], y in [0,Ly]) into a cell and a local
 * offset: cx = trunc(x/wx) clamped, then corrected by one cell if the
 * rounded local offset falls outside [0,wx); finally clamped into [0,wx). */
static void bin_axis(double x, double w, int m, int *cell, double *loc)
{
    int c = (int)(x / w);
    if (c > m - 1) c = m - 1;
    if (c < 0) c = 0;
    double l = x - (double)c * w;
    if (l < 0.0 && c > 0) { c -= 1; l = x - (double)c * w; }
    if (l >= w && c < m - 1) { c += 1; l = x - (double)c * w; }
    if (l < 0.0) l = 0.0;
    if (l >= w) l = prev_double(w);
    *cell = c;
    *loc = l;
}

/* Overlap test of every disk against the disks of its 3x3 neighbourhood, in
 * cell-local frames (same arithmetic as the sweep).  Returns #overlapping
 * ordered pairs. */
static int64_t count_overlaps_local(const oracle_t *o)
{
    int64_t bad = 0;
    for (int cy = 0; cy < o->my; ++cy)
        for (int cx = 0; cx < o->mx; ++cx) {
            int64_t c = (int64_t)cy * o->mx + cx;
            for (int i = 0; i < o->n[c]; ++i) {
                double px, py;
                slot_get(o, c, i, &px, &py);
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int ncx = (cx + dx + o->mx) % o->mx, ncy = (cy + dy + o->my) % o->my;
                        int64_t nc = (int64_t)ncy * o->mx + ncx;
                        for (int j = 0; j < o->n[nc]; ++j) {
                            if (nc == c && j == i && dx == 0 && dy == 0) continue;
                            double qx, qy;
                            slot_get(o, nc, j, &qx, &qy);
                            if (o->prec == 0) {
                                double ex = qx + (double)dx * o->wx, ey = qy + (double)dy * o->wy;
                                double ddx = px - ex, ddy = py - ey;
                                if (ddx * ddx + ddy * ddy < o->sigma * o->sigma) bad++;
                            } else {
                                float ex = (float)qx + (float)dx * o->wxf;
                                float ey = (float)qy + (float)dy * o->wyf;
                                float ddx = (float)px - ex, ddy = (float)py - ey;
                                if (overlap32(ddx, ddy, (float)(o->sigma * o->sigma))) bad++;
                            }
                        }
                    }
            }
        }
    return bad;
}

/* Place global positions xy[2N] into the cell structure (slot order within a
 * cell = ascending particle index). */
static int place(oracle_t *o, const double *xy)
{
    memset(o->n, 0, (size_t)o->C);
    for (int64_t c = 0; c < 4 * o->C; ++c) {
        if (o->prec == 0) { o->X[c] = EMPTY_SLOT; o->Y[c] = EMPTY_SLOT; }
        else { o->Xf[c] = (float)EMPTY_SLOT; o->Yf[c] = (float)EMPTY_SLOT; }
    }
    for (int64_t p = 0; p < o->N; ++p) {
        double x = xy[2 * p], y = xy[2 * p + 1];
        if (!(x >= 0.0 && x <= o->Lx && y >= 0.0 && y <= o->Ly)) return ORC_EINVAL;
        int cx, cy;
        double lx, ly;
        bin_axis(x, o->wx, o->mx, &cx, &lx);
        bin_axis(y, o->wy, o->my, &cy, &ly);
        int64_t c = (int64_t)cy * o->mx + cx;
        if (o->n[c] >= NMAX) return ORC_EOVERFLOW;
        int j = o->n[c]++;
        if (o->prec == 0) { o->X[4 * c + j] = lx; o->Y[4 * c + j] = ly; }
        else {
            float fx = (float)lx, fy = (float)ly;
            if (fx >= o->wxf) fx = prev_float(o->wxf);
            if (fy >= o->wyf) fy = prev_float(o->wyf);
            o->Xf[4 * c + j] = fx; o->Yf[4 * c + j] = fy;
        }
    }
    if (count_overlaps_local(o) != 0) return ORC_EOVERLAP;
    return ORC_OK;
}

/* Hexagonal start: choose nx*ny = N, ny even, making the row spacing Ly/ny
 * closest (in ratio) to sqrt(3)/2 times the column spacing Lx/nx. */
int orc_lattice_shape(int64_t N, double Lx, double Ly, int64_t *nx_out, int64_t *ny_out)
{
    int64_t best_nx = -1, best_ny = -1;
    double best = 0.0;
    for (int64_t ny = 2; ny <= N; ny += 2) {
        if (N % ny) continue;
        int64_t nx = N / ny;
        double cost = fabs(log((Ly / (double)ny) / ((Lx / (double)nx) * 0.86602540378443864676)));
        if (best_nx < 0 || cost < best) { best = cost; best_nx = nx; best_ny = ny; }
    }
    if (best_nx < 0) return ORC_EINVAL;
    *nx_out = best_nx; *ny_out = best_ny;
    return ORC_OK;
}

/* Lattice site p = j*nx + i at ((i + 1/2 + (j mod 2)/2) Lx/nx, (j + 1/2) Ly/ny),
 * displaced uniformly within a disk of radius 0.01 sigma (init stream of p),
 * wrapped into the box. */
int orc_lattice_positions(int64_t N, double Lx, double Ly, double sigma, uint64_t seed, double *xy)
{
    int64_t nx, ny;
    if (orc_lattice_shape(N, Lx, Ly, &nx, &ny) != ORC_OK) return ORC_EINVAL;
    double ax = Lx / (double)nx, ay = Ly / (double)ny, rj = 0.01 * sigma;
    for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
            int64_t p = j * nx + i;
            double x0 = ((double)i + 0.5 + 0.5 * (double)(j & 1)) * ax;
            double y0 = ((double)j + 0.5) * ay;
            stream_t s;
            stream_open(&s, seed, (uint32_t)p, 0xFFFFFFFEu, DOM_INIT << 28);
            double u, v;
            do {
                uint32_t a = stream_word(&s), b = stream_word(&s), c = stream_word(&s), e = stream_word(&s);
                u = sym52(a, b);
                v = sym52(c, e);
            } while (!(u * u + v * v < 1.0));
            double x = x0 + rj * u, y = y0 + rj * v;
            if (x >= Lx) x -= Lx;
            if (x < 0.0) x += Lx;
            if (y >= Ly) y -= Ly;
            if (y < 0.0) y += Ly;
            xy[2 * p] = x;
            xy[2 * p + 1] = y;
        }
    return ORC_OK;
}

int orc_create(oracle_t **out, int64_t N, double Lx, double Ly, double sigma, double d,
               int nsel, uint64_t seed, int prec)
{
    int err;
    *out = NULL;
    if (N < 2 || (N & 1)) return ORC_EINVAL;
    oracle_t *o = alloc_state(N, Lx, Ly, sigma, d, nsel, seed, prec, &err);
    if (!o) return err;
    double *xy = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    if (!xy) { orc_destroy(o); return ORC_ENOMEM; }
    err = orc_lattice_positions(N, Lx, Ly, sigma, seed, xy);
    if (err == ORC_OK) err = place(o, xy);
    free(xy);
    if (err != ORC_OK) { orc_destroy(o); return err; }
    *out = o;
    return ORC_OK;
}

int orc_create_from(oracle_t **out, int64_t N, double Lx, double Ly, double sigma, double d,
                    int nsel, uint64_t seed, int prec, const double *xy)
{
    int err;
    *out = NULL;
    oracle_t *o = alloc_state(N, Lx, Ly, sigma, d, nsel, seed, prec, &err);
    if (!o) return err;
    err = place(o, xy);
    if (err != ORC_OK) { orc_destroy(o); return err; }
    *out = o;
    return ORC_OK;
}

int orc_set_move_size(oracle_t *o, double d)
{
    if (!(d > 0) || !(d < 0.5 * o->wx) || !(d < 0.5 * o->wy)) return ORC_EINVAL;
    o->d = d;
    return ORC_OK;
}

void orc_set_balance(oracle_t *o, int shuffle_particles, int shuffle_sets)
{
    o->shuffle_particles = shuffle_particles;
    o->shuffle_sets = shuffle_sets;
}

/* ------------------------------------------------------------------------ */
/* Spatial decomposition with inactive bands (Sec. 6).  Several processors    */
/* would each own a strip of cell rows; if every cell next to another        */
/* processor's strip made moves, neighbouring processors would have to       */
/* exchange cells after every sub-sweep.  Instead the first row of every     */
/* strip is inactive during the sweep's sub-sweeps: no cell of one strip     */
/* then moves a disk next to a cell another strip moves, and strips need     */
/* each other's rows only around the grid shift.  Which cells are inactive  */
/* is fixed in the cell grid, and the grid shift moves the grid relative to */
/* the disks, so no disk stays frozen.  Strip k (0 <= k < R) is the rows     */
/* [r_k, r_{k+1}), r_k = 2 floor(k my / (2R)) (even, so every strip starts   */
/* on the same checkerboard parity; each strip has at least two rows).       */
/* ------------------------------------------------------------------------ */
int orc_strip_start(int my, int nstrips, int k)
{
    return 2 * (int)(((int64_t)k * my) / (2 * (int64_t)nstrips));
}

int orc_set_strips(oracle_t *o, int nstrips)
{
    if (nstrips < 0 || (nstrips > 0 && o->my < 2 * nstrips)) return ORC_EINVAL;
    free(o->band);
    o->band = NULL;
    o->nstrips = nstrips;
    if (nstrips == 0) return ORC_OK;
    o->band = (uint8_t *)calloc((size_t)o->my, 1);
    if (!o->band) { o->nstrips = 0; return ORC_ENOMEM; }
    for (int k = 0; k < nstrips; ++k) o->band[orc_strip_start(o->my, nstrips, k)] = 1;
    return ORC_OK;
}

/* One cell row in canonical slot order: local[(4 cx + j) 2 + {0,1}], counts[cx]
 * (unused slots read EMPTY_SLOT).  set_row replaces the row (used to hand
 * rows between the strips of a decomposed run). */
void orc_get_row(const oracle_t *o, int cy, double *local, uint8_t *counts)
{
    for (int cx = 0; cx < o->mx; ++cx) {
        int64_t c = (int64_t)cy * o->mx + cx;
        counts[cx] = o->n[c];
        for (int j = 0; j < 4; ++j) {
            double x = EMPTY_SLOT, y = EMPTY_SLOT;
            if (is_set(o, c, j)) slot_get(o, c, j, &x, &y);
            local[2 * (4 * cx + j)] = x;
            local[2 * (4 * cx + j) + 1] = y;
        }
    }
}

void orc_set_row(oracle_t *o, int cy, const double *local, const uint8_t *counts)
{
    for (int cx = 0; cx < o->mx; ++cx) {
        int64_t c = (int64_t)cy * o->mx + cx;
        o->n[c] = counts[cx];
        for (int j = 0; j < 4; ++j) {
            double x = j < counts[cx] ? local[2 * (4 * cx + j)] : EMPTY_SLOT;
            double y = j < counts[cx] ? local[2 * (4 * cx + j) + 1] : EMPTY_SLOT;
            if (o->prec == 0) { o->X[4 * c + j] = x; o->Y[4 * c + j] = y; }
            else { o->Xf[4 * c + j] = (float)x; o->Yf[4 * c + j] = (float)y; }
        }
    }
}

int orc_set_allow_leave(oracle_t *o, int allow)
{
    o->allow_leave = allow;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Sweep-level draws (Alg. 1): set order by Fisher-Yates, shift direction f  */
/* in {+x,-x,+y,-y}, shift distance d ~ U(0, w/2) along f's axis.            */
/* ------------------------------------------------------------------------ */
typedef struct { int perm[4]; int fdir; double ds; } draws_t;

static void sweep_draws(uint64_t seed, uint32_t sweep, double wx, double wy, draws_t *r)
{
    stream_t s;
    stream_open(&s, seed, sweep, 0xFFFFFFFFu, DOM_SWEEP << 28);
    for (int q = 0; q < 4; ++q) r->perm[q] = q;
    for (int j = 3; j >= 1; --j) {
        int k = (int)stream_bounded(&s, (uint32_t)(j + 1));
        int t = r->perm[j]; r->perm[j] = r->perm[k]; r->perm[k] = t;
    }
    r->fdir = (int)stream_bounded(&s, 4u);
    uint32_t hi = stream_word(&s), lo = stream_word(&s);
    double w = (r->fdir >> 1) ? wy : wx;
    r->ds = unif53(hi, lo) * (0.5 * w);
}

static void shift_draws(uint64_t seed, uint32_t index, double wx, double wy, draws_t *r)
{
    stream_t s;
    stream_open(&s, seed, index, 0xFFFFFFFFu, DOM_SHIFT << 28);
    for (int q = 0; q < 4; ++q) r->perm[q] = q;
    r->fdir = (int)stream_bounded(&s, 4u);
    uint32_t hi = stream_word(&s), lo = stream_word(&s);
    double w = (r->fdir >> 1) ? wy : wx;
    r->ds = unif53(hi, lo) * (0.5 * w);
}

void orc_sweep_draws(uint64_t seed, uint32_t sweep, double wx, double wy, int32_t perm[4],
                     int32_t *fdir, double *ds)
{
    draws_t r;
    sweep_draws(seed, sweep, wx, wy, &r);
    for (int q = 0; q < 4; ++q) perm[q] = r.perm[q];
    *fdir = r.fdir;
    *ds = r.ds;
}


/* ------------------------------------------------------------------------ */
/* Per-cell random draws of a sub-sweep (Alg. 1: shuffle, trial directions). */
/*                                                                          */
/* One cell update (sweep s, set Q, canonical cell c) reads its trial       */
/* stream T = (s, c, (1<<28)|(Q<<24)) and, for binary64 shuffles or a      */
/* rejected binary32 shuffle draw, its shuffle stream                      */
/* S = (s, c, (0<<28)|(Q<<24)).  The draws do not depend on positions, so  */
/* they are all taken before the trials.                                    */
/*  - Shuffle (n >= 2): one integer k uniform in [0, n!) decoded as the    */
/*    Fisher-Yates swap sequence (mixed radix), i.e. a uniform random      */
/*    permutation of the cell's n disks.                                   */
/*  - Directions: attempts (u,v) uniform in (-1,1)^2, kept when inside the */
/*    unit disk; trial t uses the t-th kept attempt.                       */
/* binary64: k by 32-bit Lemire on the words of S; attempt a = block a of T */
/*   with u = sym52(w0,w1), v = sym52(w2,w3), kept when u*u + v*v < 1.      */
/* binary32: block b of T is cut into six 21-bit fields; k by 21-bit        */
/*   Lemire on field 0 of block 0 (if rejected: 32-bit Lemire on S); the   */
/*   attempts are the field pairs (2,3),(4,5) of block 0, then (0,1),(2,3), */
/*   (4,5) of blocks 1, 2, ...; u = sym21, kept when fmaf(u,u,v*v) < 1.    */
/* ------------------------------------------------------------------------ */

static const uint32_t kFactorial[5] = {1u, 1u, 2u, 6u, 24u};

/* Field j (0..5) = bits [21j, 21j+21) of w0 + 2^32 w1 + 2^64 w2 + 2^96 w3. */
static void fields21(const uint32_t w[4], uint32_t f[6])
{
    for (int j = 0; j < 6; ++j) {
        int bit = 21 * j, word = bit / 32;
        uint64_t both = (uint64_t)w[word];
        if (word + 1 < 4) both |= (uint64_t)w[word + 1] << 32;
        f[j] = (uint32_t)((both >> (bit % 32)) & 0x1FFFFFu);
    }
}

/* Lemire's method on a 21-bit field: value floor(f*range / 2^21), rejected
 * when the low 21 bits of f*range fall below 2^21 mod range. */
static int lemire21(uint32_t f, uint32_t range, uint32_t *value)
{
    uint32_t threshold = (1u << 21) % range;
    uint32_t m = f * range;
    *value = m >> 21;
    return (m & 0x1FFFFFu) >= threshold;
}

/* Odd multiples of 2^-21 in (-1,1) from a 21-bit field. */
static float sym21(uint32_t f)
{
    int32_t m = (int32_t)(2 * f + 1) - (1 << 21);
    return (float)m * 0x1p-21f;
}

/* Fisher-Yates decode of k in [0, n!): for j = n-1 down to 1 swap slots j and
 * k mod (j+1), then k /= (j+1).  perm[j] = old slot that now sits in slot j. */
static void decode_perm(int n, uint32_t k, int perm[4])
{
    for (int j = 0; j < 4; ++j) perm[j] = j;
    for (int j = n - 1; j >= 1; --j) {
        int r = (int)(k % (uint32_t)(j + 1));
        k /= (uint32_t)(j + 1);
        int t = perm[j]; perm[j] = perm[r]; perm[r] = t;
    }
}

static void philox_block(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t b, uint32_t w[4])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {c0, c1, c2, b};
    orc_philox(ctr, key, w);
}

/* binary64 draws of one cell update. */
static void cell_draws64(uint64_t seed, uint32_t sweep, uint32_t cell, int Q, int n, int shuffle, int nsel,
                         int perm[4], double *U, double *V)
{
    const uint32_t setbits = (uint32_t)Q << 24;
    for (int j = 0; j < 4; ++j) perm[j] = j;
    if (shuffle && n >= 2) {
        stream_t s;
        stream_open(&s, seed, sweep, cell, (DOM_SHUFFLE << 28) | setbits);
        decode_perm(n, stream_bounded(&s, kFactorial[n]), perm);
    }
    uint32_t block = 0;
    for (int t = 0; t < nsel;) {
        uint32_t w[4];
        philox_block(seed, sweep, cell, (DOM_TRIAL << 28) | setbits, block++, w);
        double u = sym52(w[0], w[1]), v = sym52(w[2], w[3]);
        if (u * u + v * v < 1.0) { U[t] = u; V[t] = v; ++t; }
    }
}

/* binary32 draws of one cell update. */
static void cell_draws32(uint64_t seed, uint32_t sweep, uint32_t cell, int Q, int n, int shuffle, int nsel,
                         int perm[4], float *U, float *V)
{
    const uint32_t setbits = (uint32_t)Q << 24;
    uint32_t w[4], f[6];
    philox_block(seed, sweep, cell, (DOM_TRIAL << 28) | setbits, 0, w);
    fields21(w, f);
    for (int j = 0; j < 4; ++j) perm[j] = j;
    if (shuffle && n >= 2) {
        uint32_t k;
        if (!lemire21(f[0], kFactorial[n], &k)) {
            stream_t s;
            stream_open(&s, seed, sweep, cell, (DOM_SHUFFLE << 28) | setbits);
            k = stream_bounded(&s, kFactorial[n]);
        }
        decode_perm(n, k, perm);
    }
    uint32_t block = 0;
    int pair = 1;
    for (int t = 0; t < nsel;) {
        if (pair == 3) {
            philox_block(seed, sweep, cell, (DOM_TRIAL << 28) | setbits, ++block, w);
            fields21(w, f);
            pair = 0;
        }
        float u = sym21(f[2 * pair]), v = sym21(f[2 * pair + 1]);
        ++pair;
        if (fmaf(u, u, v * v) < 1.0f) { U[t] = u; V[t] = v; ++t; }
    }
}

/* Test hooks: direction of trial t (shuffle off, so independent of n) and
 * the permutation of an n-disk cell, for cells 0..ncells-1. */
void orc_displacements(uint64_t seed, uint32_t sweep, int Q, int t, int prec, int64_t ncells, double *uv)
{
    int perm[4];
    double *U = (double *)malloc(sizeof(double) * (size_t)(t + 1));
    double *V = (double *)malloc(sizeof(double) * (size_t)(t + 1));
    float *Uf = (float *)malloc(sizeof(float) * (size_t)(t + 1));
    float *Vf = (float *)malloc(sizeof(float) * (size_t)(t + 1));
    for (int64_t c = 0; c < ncells; ++c) {
        if (prec == 0) {
            cell_draws64(seed, sweep, (uint32_t)c, Q, 1, 0, t + 1, perm, U, V);
            uv[2 * c] = U[t]; uv[2 * c + 1] = V[t];
        } else {
            cell_draws32(seed, sweep, (uint32_t)c, Q, 1, 0, t + 1, perm, Uf, Vf);
            uv[2 * c] = Uf[t]; uv[2 * c + 1] = Vf[t];
        }
    }
    free(U); free(V); free(Uf); free(Vf);
}

void orc_shuffles(uint64_t seed, uint32_t sweep, int Q, int n, int prec, int64_t ncells, int32_t *perms)
{
    double U[1], V[1];
    float Uf[1], Vf[1];
    for (int64_t c = 0; c < ncells; ++c) {
        int p[4];
        if (prec == 0) cell_draws64(seed, sweep, (uint32_t)c, Q, n, 1, 1, p, U, V);
        else cell_draws32(seed, sweep, (uint32_t)c, Q, n, 1, 1, p, Uf, Vf);
        for (int j = 0; j < 4; ++j) perms[4 * c + j] = p[j];
    }
}

/* Exhaustive 21-bit Lemire counts (range <= 24): counts[v] = #fields -> v. */
void orc_lemire21_exhaustive(uint32_t range, uint64_t *counts)
{
    memset(counts, 0, sizeof(uint64_t) * range);
    for (uint32_t f = 0; f < (1u << 21); ++f) {
        uint32_t v;
        if (lemire21(f, range, &v)) counts[v] += 1;
    }
}

float orc_sym21(uint32_t f) { return sym21(f); }

void orc_fields21(const uint32_t w[4], uint32_t f[6]) { fields21(w, f); }

void orc_decode_perm(int n, uint32_t k, int32_t out[4])
{
    int p[4];
    decode_perm(n, k, p);
    for (int j = 0; j < 4; ++j) out[j] = p[j];
}

/* Slot visited by trial t of a cell holding n disks: t mod n (Alg. 1).      */
static int visit_slot(int t, int n) { return t % n; }

void orc_visit_sequence(int n, int nsel, int32_t *seq)
{
    for (int t = 0; t < nsel; ++t) seq[t] = visit_slot(t, n);
}

/* ------------------------------------------------------------------------ */
/* Negative control of Sec. 2.4 item 1: a disk whose trial position lies     */
/* outside its cell moves into the neighbouring cell that contains it, if   */
/* it overlaps no disk of that cell's 3x3 neighbourhood and the cell has a  */
/* free slot.  It is appended there and removed from its own cell (the      */
/* remaining slots close up; the cell's visit sequence continues with the   */
/* new count).  Serial order only.  Returns 1 moved, 0 overlap, 2 no slot.  */
/* ------------------------------------------------------------------------ */
static int leave_cell64(oracle_t *o, int cx, int cy, int i, double nx, double ny)
{
    int ex = nx < 0.0 ? -1 : (nx >= o->wx ? 1 : 0);
    int ey = ny < 0.0 ? -1 : (ny >= o->wy ? 1 : 0);
    double lx = nx - (double)ex * o->wx, ly = ny - (double)ey * o->wy;
    if (lx < 0.0) lx = 0.0;
    if (lx >= o->wx) lx = prev_double(o->wx);
    if (ly < 0.0) ly = 0.0;
    if (ly >= o->wy) ly = prev_double(o->wy);
    int dcx = (cx + ex + o->mx) % o->mx, dcy = (cy + ey + o->my) % o->my;
    int64_t c = (int64_t)cy * o->mx + cx, dc = (int64_t)dcy * o->mx + dcx;
    if (o->n[dc] >= NMAX) return 2;
    const double sig2 = o->sigma * o->sigma;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            int ncx = (dcx + dx + o->mx) % o->mx, ncy = (dcy + dy + o->my) % o->my;
            int64_t nc = (int64_t)ncy * o->mx + ncx;
            for (int j = 0; j < o->n[nc]; ++j) {
                if (nc == c && j == i) continue;
                double ddx = lx - (o->X[4 * nc + j] + (double)dx * o->wx);
                double ddy = ly - (o->Y[4 * nc + j] + (double)dy * o->wy);
                if (ddx * ddx + ddy * ddy < sig2) return 0;
            }
        }
    int k = o->n[dc]++;
    o->X[4 * dc + k] = lx;
    o->Y[4 * dc + k] = ly;
    for (int j = i; j + 1 < o->n[c]; ++j) {
        o->X[4 * c + j] = o->X[4 * c + j + 1];
        o->Y[4 * c + j] = o->Y[4 * c + j + 1];
    }
    o->n[c]--;
    o->X[4 * c + o->n[c]] = EMPTY_SLOT;
    o->Y[4 * c + o->n[c]] = EMPTY_SLOT;
    return 1;
}

/* The same negative control in the binary32 mode: binary32 widths, the
 * binary32 overlap predicate and binary32 re-expression in the new cell. */
static int leave_cell32(oracle_t *o, int cx, int cy, int i, float nx, float ny)
{
    int ex = nx < 0.0f ? -1 : (nx >= o->wxf ? 1 : 0);
    int ey = ny < 0.0f ? -1 : (ny >= o->wyf ? 1 : 0);
    float lx = nx - (float)ex * o->wxf, ly = ny - (float)ey * o->wyf;
    if (lx < 0.0f) lx = 0.0f;
    if (lx >= o->wxf) lx = prev_float(o->wxf);
    if (ly < 0.0f) ly = 0.0f;
    if (ly >= o->wyf) ly = prev_float(o->wyf);
    int dcx = (cx + ex + o->mx) % o->mx, dcy = (cy + ey + o->my) % o->my;
    int64_t c = (int64_t)cy * o->mx + cx, dc = (int64_t)dcy * o->mx + dcx;
    if (o->n[dc] >= NMAX) return 2;
    const float sig2 = (float)(o->sigma * o->sigma);
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            int ncx = (dcx + dx + o->mx) % o->mx, ncy = (dcy + dy + o->my) % o->my;
            int64_t nc = (int64_t)ncy * o->mx + ncx;
            for (int j = 0; j < o->n[nc]; ++j) {
                if (nc == c && j == i) continue;
                float ddx = lx - (o->Xf[4 * nc + j] + (float)dx * o->wxf);
                float ddy = ly - (o->Yf[4 * nc + j] + (float)dy * o->wyf);
                if (overlap32(ddx, ddy, sig2)) return 0;
            }
        }
    int k = o->n[dc]++;
    o->Xf[4 * dc + k] = lx;
    o->Yf[4 * dc + k] = ly;
    for (int j = i; j + 1 < o->n[c]; ++j) {
        o->Xf[4 * c + j] = o->Xf[4 * c + j + 1];
        o->Yf[4 * c + j] = o->Yf[4 * c + j + 1];
    }
    o->n[c]--;
    o->Xf[4 * c + o->n[c]] = (float)EMPTY_SLOT;
    o->Yf[4 * c + o->n[c]] = (float)EMPTY_SLOT;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* One cell update of a sub-sweep (Alg. 1, Alg. 2)                          */
/* ------------------------------------------------------------------------ */

static void cell_update64(oracle_t *o, uint32_t sweep, int Q, int cx, int cy, uint64_t acc[4])
{
    int64_t c = (int64_t)cy * o->mx + cx;
    int n = o->n[c];
    if (n == 0) return;
    double *X = o->X + 4 * c, *Y = o->Y + 4 * c;
    int perm[4];
    double U[256], V[256];
    cell_draws64(o->seed, sweep, (uint32_t)c, Q, n, o->shuffle_particles, o->nsel, perm, U, V);
    /* shuffle the cell's particles (Alg. 1) */
    double tx[4], ty[4];
    for (int j = 0; j < n; ++j) { tx[j] = X[perm[j]]; ty[j] = Y[perm[j]]; }
    for (int j = 0; j < n; ++j) { X[j] = tx[j]; Y[j] = ty[j]; }
    const double sig2 = o->sigma * o->sigma;
    for (int t = 0; t < o->nsel; ++t) {
        int i = visit_slot(t, n);
        double nx = X[i] + o->d * U[t];
        double ny = Y[i] + o->d * V[t];
        acc[0]++;
        if (!(nx >= 0.0 && nx < o->wx && ny >= 0.0 && ny < o->wy)) {
            if (!o->allow_leave) { acc[2]++; continue; }
            int r = leave_cell64(o, cx, cy, i, nx, ny);
            if (r == 1) {
                acc[1]++;
                n = o->n[c];
                if (n == 0) break;
            } else {
                acc[r == 0 ? 3 : 2]++;
            }
            continue;
        }
        int overlap = 0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double ddx = nx - X[j], ddy = ny - Y[j];
            if (ddx * ddx + ddy * ddy < sig2) overlap = 1;
        }
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0) continue;
                int ncx = (cx + dx + o->mx) % o->mx, ncy = (cy + dy + o->my) % o->my;
                int64_t nc = (int64_t)ncy * o->mx + ncx;
                double sx = (double)dx * o->wx, sy = (double)dy * o->wy;
                for (int j = 0; j < o->n[nc]; ++j) {
                    double ex = o->X[4 * nc + j] + sx, ey = o->Y[4 * nc + j] + sy;
                    double ddx = nx - ex, ddy = ny - ey;
                    if (ddx * ddx + ddy * ddy < sig2) overlap = 1;
                }
            }
        if (overlap) { acc[3]++; continue; }
        X[i] = nx;
        Y[i] = ny;
        acc[1]++;
    }
}

static void cell_update32(oracle_t *o, uint32_t sweep, int Q, int cx, int cy, uint64_t acc[4])
{
    int64_t c = (int64_t)cy * o->mx + cx;
    int n = o->n[c];
    if (n == 0) return;
    float *X = o->Xf + 4 * c, *Y = o->Yf + 4 * c;
    int perm[4];
    float U[256], V[256];
    cell_draws32(o->seed, sweep, (uint32_t)c, Q, n, o->shuffle_particles, o->nsel, perm, U, V);
    float tx[4], ty[4];
    for (int j = 0; j < n; ++j) { tx[j] = X[perm[j]]; ty[j] = Y[perm[j]]; }
    for (int j = 0; j < n; ++j) { X[j] = tx[j]; Y[j] = ty[j]; }
    const float sig2 = (float)(o->sigma * o->sigma);
    const float df = (float)o->d;
    for (int t = 0; t < o->nsel; ++t) {
        int i = visit_slot(t, n);
        float nx = fmaf(df, U[t], X[i]);
        float ny = fmaf(df, V[t], Y[i]);
        acc[0]++;
        if (!(nx >= 0.0f && nx < o->wxf && ny >= 0.0f && ny < o->wyf)) {
            if (!o->allow_leave) { acc[2]++; continue; }
            int r = leave_cell32(o, cx, cy, i, nx, ny);
            if (r == 1) {
                acc[1]++;
                n = o->n[c];
                if (n == 0) break;
            } else {
                acc[r == 0 ? 3 : 2]++;
            }
            continue;
        }
        int overlap = 0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            float ddx = nx - X[j], ddy = ny - Y[j];
            if (overlap32(ddx, ddy, sig2)) overlap = 1;
        }
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0) continue;
                int ncx = (cx + dx + o->mx) % o->mx, ncy = (cy + dy + o->my) % o->my;
                int64_t nc = (int64_t)ncy * o->mx + ncx;
                float sx = (float)dx * o->wxf, sy = (float)dy * o->wyf;
                for (int j = 0; j < o->n[nc]; ++j) {
                    float ex = o->Xf[4 * nc + j] + sx, ey = o->Yf[4 * nc + j] + sy;
                    float ddx = nx - ex, ddy = ny - ey;
                    if (overlap32(ddx, ddy, sig2)) overlap = 1;
                }
            }
        if (overlap) { acc[3]++; continue; }
        X[i] = nx;
        Y[i] = ny;
        acc[1]++;
    }
}

/* All cells of checkerboard set Q (Eq. 1: Q = (cx mod 2) + 2 (cy mod 2)),
 * i.e. the cell updates of one set in Alg. 1.  Cells of one set are
 * independent. */
static void subsweep(oracle_t *o, uint32_t sweep, int Q)
{
    int qx = Q & 1, qy = Q >> 1;
    uint64_t t0 = 0, t1 = 0, t2 = 0, t3 = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(+ : t0, t1, t2, t3) if (!o->allow_leave && o->C >= 4096)
#endif
    for (int cy = qy; cy < o->my; cy += 2) {
        uint64_t acc[4] = {0, 0, 0, 0};
        if (o->band && o->band[cy]) continue;   /* inactive band row (Sec. 6) */
        for (int cx = qx; cx < o->mx; cx += 2) {
            if (o->prec == 0) cell_update64(o, sweep, Q, cx, cy, acc);
            else cell_update32(o, sweep, Q, cx, cy, acc);
        }
        t0 += acc[0]; t1 += acc[1]; t2 += acc[2]; t3 += acc[3];
    }
    o->cnt[0] += t0; o->cnt[1] += t1; o->cnt[2] += t2; o->cnt[3] += t3;
}

/* binary32 value stored for a remapped binary64 coordinate v >= 0 of a cell
 * of binary32 width wf: v rounded to nearest, clamped below wf (a value just
 * under the edge may round onto it). */
static float store32(double v, float wf)
{
    float f = (float)v;
    if (f >= wf) f = prev_float(wf);
    if (f < 0.0f) f = 0.0f;
    return f;
}

/* ------------------------------------------------------------------------ */
/* Cell shift (Alg. 4): translate every disk by -f*ds.  New cell c keeps the */
/* disks of old c that stay inside it (old slot order), then takes the disks */
/* of old c+f that leave c+f, re-expressed in c's frame.  The ownership test */
/* is the same expression in both places, so no disk is lost (Sec. 3.2).    */
/* ------------------------------------------------------------------------ */
static int shift_cells(oracle_t *o, int fdir, double ds)
{
    int ax = fdir >> 1;
    int sgn = (fdir & 1) ? -1 : 1;
    int64_t C = o->C;
    uint8_t *nn = (uint8_t *)calloc((size_t)C, 1);
    int overflow = 0;
    if (o->prec == 0) {
        double w = ax ? o->wy : o->wx;
        double sd = (double)sgn * ds;
        double sw = (double)sgn * w;
        double *NX = (double *)malloc(sizeof(double) * 4 * (size_t)C);
        double *NY = (double *)malloc(sizeof(double) * 4 * (size_t)C);
        for (int cy = 0; cy < o->my; ++cy)
            for (int cx = 0; cx < o->mx; ++cx) {
                int64_t c = (int64_t)cy * o->mx + cx;
                int ncx = ax ? cx : (cx + sgn + o->mx) % o->mx;
                int ncy = ax ? (cy + sgn + o->my) % o->my : cy;
                int64_t nb = (int64_t)ncy * o->mx + ncx;
                double ox[8], oy[8];
                int k = 0;
                for (int j = 0; j < o->n[c]; ++j) {
                    double px = o->X[4 * c + j], py = o->Y[4 * c + j];
                    double dp = (ax ? py : px) - sd;
                    if (dp >= 0.0 && dp < w) {
                        ox[k] = ax ? px : dp; oy[k] = ax ? dp : py; k++;
                    }
                }
                for (int j = 0; j < o->n[nb]; ++j) {
                    double px = o->X[4 * nb + j], py = o->Y[4 * nb + j];
                    double dp = (ax ? py : px) - sd;
                    if (!(dp >= 0.0 && dp < w)) {
                        double v = dp + sw;
                        if (v >= w) v = prev_double(w);
                        if (v < 0.0) v = 0.0;
                        ox[k] = ax ? px : v; oy[k] = ax ? v : py; k++;
                    }
                }
                if (k > NMAX) { overflow = 1; k = NMAX; }
                nn[c] = (uint8_t)k;
                for (int j = 0; j < 4; ++j) {
                    NX[4 * c + j] = j < k ? ox[j] : EMPTY_SLOT;
                    NY[4 * c + j] = j < k ? oy[j] : EMPTY_SLOT;
                }
            }
        free(o->X); free(o->Y);
        o->X = NX; o->Y = NY;
        if (ax) o->Oy += sd; else o->Ox += sd;
    } else {
        /* binary32 positions, binary64 remap: the translation x - sd and the
         * ownership test are evaluated in binary64 on the binary32 cell
         * width W (exact in binary64), and only the result is rounded to
         * binary32 (then clamped below the cell's upper edge) */
        float wf = ax ? o->wyf : o->wxf;
        double W = (double)wf;
        double sd = (double)sgn * ds;
        double sW = (double)sgn * W;
        float *NX = (float *)malloc(sizeof(float) * 4 * (size_t)C);
        float *NY = (float *)malloc(sizeof(float) * 4 * (size_t)C);
        for (int cy = 0; cy < o->my; ++cy)
            for (int cx = 0; cx < o->mx; ++cx) {
                int64_t c = (int64_t)cy * o->mx + cx;
                int ncx = ax ? cx : (cx + sgn + o->mx) % o->mx;
                int ncy = ax ? (cy + sgn + o->my) % o->my : cy;
                int64_t nb = (int64_t)ncy * o->mx + ncx;
                float ox[8], oy[8];
                int k = 0;
                for (int j = 0; j < o->n[c]; ++j) {
                    float px = o->Xf[4 * c + j], py = o->Yf[4 * c + j];
                    double dp = (double)(ax ? py : px) - sd;
                    if (dp >= 0.0 && dp < W) {
                        float v = store32(dp, wf);
                        ox[k] = ax ? px : v; oy[k] = ax ? v : py; k++;
                    }
                }
                for (int j = 0; j < o->n[nb]; ++j) {
                    float px = o->Xf[4 * nb + j], py = o->Yf[4 * nb + j];
                    double dp = (double)(ax ? py : px) - sd;
                    if (!(dp >= 0.0 && dp < W)) {
                        float v = store32(dp + sW, wf);
                        ox[k] = ax ? px : v; oy[k] = ax ? v : py; k++;
                    }
                }
                if (k > NMAX) { overflow = 1; k = NMAX; }
                nn[c] = (uint8_t)k;
                for (int j = 0; j < 4; ++j) {
                    NX[4 * c + j] = j < k ? ox[j] : (float)EMPTY_SLOT;
                    NY[4 * c + j] = j < k ? oy[j] : (float)EMPTY_SLOT;
                }
            }
        free(o->Xf); free(o->Yf);
        o->Xf = NX; o->Yf = NY;
        if (ax) o->Oy += sd; else o->Ox += sd;
    }
    free(o->n);
    o->n = nn;
    return overflow ? ORC_EOVERFLOW : ORC_OK;
}

/* n full sweeps (Alg. 1). */
int orc_sweep(oracle_t *o, int64_t nsweeps)
{
    for (int64_t k = 0; k < nsweeps; ++k) {
        uint32_t sweep = (uint32_t)o->sweep;
        draws_t r;
        sweep_draws(o->seed, sweep, o->wx, o->wy, &r);
        for (int q = 0; q < 4; ++q) {
            int Q = o->shuffle_sets ? r.perm[q] : q;
            subsweep(o, sweep, Q);
        }
        int err = shift_cells(o, r.fdir, r.ds);
        o->sweep += 1;
        if (err != ORC_OK) return err;
    }
    return ORC_OK;
}

/* One sweep in two phases, as a decomposed run performs it (Sec. 6): phase 0
 * the four sub-sweeps of sweep o->sweep, phase 1 its grid shift (then the
 * sweep counter advances).  Phase 0 then phase 1 equals orc_sweep(o, 1). */
int orc_sweep_phase(oracle_t *o, int phase)
{
    uint32_t sweep = (uint32_t)o->sweep;
    draws_t r;
    sweep_draws(o->seed, sweep, o->wx, o->wy, &r);
    if (phase == 0) {
        for (int q = 0; q < 4; ++q) subsweep(o, sweep, o->shuffle_sets ? r.perm[q] : q);
        return ORC_OK;
    }
    int err = shift_cells(o, r.fdir, r.ds);
    o->sweep += 1;
    return err;
}

/* One explicit extra shift drawn from its own stream (index = #shifts so far). */
int orc_shift(oracle_t *o)
{
    draws_t r;
    shift_draws(o->seed, (uint32_t)o->shifts, o->wx, o->wy, &r);
    o->shifts += 1;
    return shift_cells(o, r.fdir, r.ds);
}

/* One sub-sweep of set Q with the draws of sweep index `sweep` (tests only). */
void orc_subsweep(oracle_t *o, uint32_t sweep, int Q) { subsweep(o, sweep, Q); }

/* ------------------------------------------------------------------------ */
/* Accessors                                                                 */
/* ------------------------------------------------------------------------ */
void orc_info(const oracle_t *o, int32_t *mx, int32_t *my, double *wx, double *wy,
              uint64_t *sweep, uint64_t *shifts)
{
    *mx = o->mx; *my = o->my; *wx = o->wx; *wy = o->wy;
    *sweep = o->sweep; *shifts = o->shifts;
}

void orc_counters(const oracle_t *o, uint64_t out[4])
{
    for (int k = 0; k < 4; ++k) out[k] = o->cnt[k];
}

void orc_origin(const oracle_t *o, double out[2]) { out[0] = o->Ox; out[1] = o->Oy; }

/* Raw state in canonical order: local[(4c+j)*2 + {0,1}], counts[c]; unused
 * slots read EMPTY_SLOT. */
void orc_state(const oracle_t *o, double *local, uint8_t *counts)
{
    for (int64_t c = 0; c < o->C; ++c) {
        counts[c] = o->n[c];
        for (int j = 0; j < 4; ++j) {
            double x = EMPTY_SLOT, y = EMPTY_SLOT;
            if (is_set(o, c, j)) slot_get(o, c, j, &x, &y);
            local[2 * (4 * c + j)] = x;
            local[2 * (4 * c + j) + 1] = y;
        }
    }
}

/* Global coordinates in canonical (cell, slot) order:
 *   g = O + (cell*w + local), wrapped into [0, m*w) by g - L floor(g/L),
 * with w the mode's cell width (binary32 widths in FP32 mode). */
void orc_positions(const oracle_t *o, double *xy)
{
    double wx = o->prec == 0 ? o->wx : (double)o->wxf;
    double wy = o->prec == 0 ? o->wy : (double)o->wyf;
    double Lx = o->prec == 0 ? o->Lx : (double)o->mx * wx;
    double Ly = o->prec == 0 ? o->Ly : (double)o->my * wy;
    int64_t p = 0;
    for (int cy = 0; cy < o->my; ++cy)
        for (int cx = 0; cx < o->mx; ++cx) {
            int64_t c = (int64_t)cy * o->mx + cx;
            for (int j = 0; j < o->n[c]; ++j) {
                double lx, ly;
                slot_get(o, c, j, &lx, &ly);
                double gx = o->Ox + ((double)cx * wx + lx);
                double gy = o->Oy + ((double)cy * wy + ly);
                gx = gx - Lx * floor(gx / Lx);
                gy = gy - Ly * floor(gy / Ly);
                xy[2 * p] = gx;
                xy[2 * p + 1] = gy;
                p++;
            }
        }
}

/* ------------------------------------------------------------------------ */
/* Contact histogram (Sec. 4): ordered pairs (i, j != i) at distance r with  */
/* sigma <= r < sigma + nbins*dr, bin floor((r - sigma)/dr).  Distances are  */
/* taken in cell-local frames over the 5x5 cell neighbourhood (w >= sigma,   */
/* so two rings reach past sigma + c for c <= sigma), in binary64.          */
/* ------------------------------------------------------------------------ */
/* Bin of a squared distance r2: bin b covers [E_b, E_{b+1}) with the squared
 * edges E_k = e_k * e_k, e_k = sigma + k*dr (each product and sum rounded
 * once in binary64); -1 outside [E_0, E_nbins). */
static int bin_of_r2(double r2, double sigma, double dr, int nbins)
{
    double e0 = sigma;
    if (!(r2 >= e0 * e0)) return -1;
    double en = sigma + (double)nbins * dr;
    if (!(r2 < en * en)) return -1;
    int b = 0;
    for (int k = 1; k < nbins; ++k) {
        double e = sigma + (double)k * dr;
        if (r2 >= e * e) b = k;
    }
    return b;
}

void orc_edges2(double sigma, double dr, int nbins, double *E)
{
    for (int k = 0; k <= nbins; ++k) {
        double e = sigma + (double)k * dr;
        E[k] = e * e;
    }
}

void orc_histogram(const oracle_t *o, int nbins, double dr, uint64_t *hist)
{
    memset(hist, 0, sizeof(uint64_t) * (size_t)nbins);
    double wx = o->prec == 0 ? o->wx : (double)o->wxf;
    double wy = o->prec == 0 ? o->wy : (double)o->wyf;
    double sigma = o->sigma;
    for (int cy = 0; cy < o->my; ++cy)
        for (int cx = 0; cx < o->mx; ++cx) {
            int64_t c = (int64_t)cy * o->mx + cx;
            for (int i = 0; i < o->n[c]; ++i) {
                double px, py;
                slot_get(o, c, i, &px, &py);
                for (int dy = -2; dy <= 2; ++dy)
                    for (int dx = -2; dx <= 2; ++dx) {
                        int ncx = ((cx + dx) % o->mx + o->mx) % o->mx;
                        int ncy = ((cy + dy) % o->my + o->my) % o->my;
                        int64_t nc = (int64_t)ncy * o->mx + ncx;
                        double sx = (double)dx * wx, sy = (double)dy * wy;
                        for (int j = 0; j < o->n[nc]; ++j) {
                            if (dx == 0 && dy == 0 && j == i) continue;
                            double qx, qy;
                            slot_get(o, nc, j, &qx, &qy);
                            double ddx = px - (qx + sx), ddy = py - (qy + sy);
                            int b = bin_of_r2(ddx * ddx + ddy * ddy, sigma, dr, nbins);
                            if (b >= 0) hist[b] += 1;
                        }
                    }
            }
        }
}

/* ------------------------------------------------------------------------ */
/* Bond-orientational order psi_6 (the "average orientational order           */
/* parameter" whose autocorrelation time Sec. 3.3 minimises).  Reading: the   */
/* neighbours k of disk j are the other disks closer than r_cut (given by the */
/* caller, at most two cell widths); psi_6(j) = (1/n_j) sum_k (z_jk/|z_jk|)^6 */
/* with z_jk = dx + i dy, the separation in cell-local terms as in the        */
/* histogram; psi_6(j) = 0 without neighbours.  (z/|z|)^6 = z^6 / (|z|^2)^3:  */
/* complex products and one division per pair, in the order written.         */
/* out[0] + i out[1] = sum_j psi_6(j), out[2] = sum_j |psi_6(j)|,             */
/* out[3] = sum_j n_j; psi (nullable) receives psi_6 of every slot in the     */
/* canonical layout psi[(4c + j)*2 + k], k = 0 real, 1 imaginary (0 where a   */
/* slot is unused).                                                            */
/* ------------------------------------------------------------------------ */
void orc_psi6(const oracle_t *o, double rcut, double out[4], double *psi)
{
    const double wx = o->prec == 0 ? o->wx : (double)o->wxf;
    const double wy = o->prec == 0 ? o->wy : (double)o->wyf;
    const double rc2 = rcut * rcut;
    double sre = 0.0, sim = 0.0, sabs = 0.0, snb = 0.0;
    if (psi) memset(psi, 0, sizeof(double) * 8 * (size_t)o->mx * (size_t)o->my);
    for (int cy = 0; cy < o->my; ++cy)
        for (int cx = 0; cx < o->mx; ++cx) {
            int64_t c = (int64_t)cy * o->mx + cx;
            for (int i = 0; i < o->n[c]; ++i) {
                double px, py;
                slot_get(o, c, i, &px, &py);
                double are = 0.0, aim = 0.0;
                int nb = 0;
                for (int dy = -2; dy <= 2; ++dy)
                    for (int dx = -2; dx <= 2; ++dx) {
                        int ncx = ((cx + dx) % o->mx + o->mx) % o->mx;
                        int ncy = ((cy + dy) % o->my + o->my) % o->my;
                        int64_t nc = (int64_t)ncy * o->mx + ncx;
                        double sx = (double)dx * wx, sy = (double)dy * wy;
                        for (int j = 0; j < o->n[nc]; ++j) {
                            if (dx == 0 && dy == 0 && j == i) continue;
                            double qx, qy;
                            slot_get(o, nc, j, &qx, &qy);
                            double ddx = px - (qx + sx), ddy = py - (qy + sy);
                            double r2 = ddx * ddx + ddy * ddy;
                            if (!(r2 < rc2)) continue;
                            double ar = ddx * ddx - ddy * ddy, ai = 2.0 * (ddx * ddy);   /* z^2 */
                            double br = ar * ddx - ai * ddy, bi = ar * ddy + ai * ddx;   /* z^3 */
                            double cr = br * br - bi * bi, ci = 2.0 * (br * bi);         /* z^6 */
                            double r6 = (r2 * r2) * r2;
                            are += cr / r6;
                            aim += ci / r6;
                            nb += 1;
                        }
                    }
                if (nb > 0) {
                    double pr = are / (double)nb, pi = aim / (double)nb;
                    sre += pr;
                    sim += pi;
                    sabs += sqrt(pr * pr + pi * pi);
                    if (psi) { psi[(4 * c + i) * 2] = pr; psi[(4 * c + i) * 2 + 1] = pi; }
                }
                snb += (double)nb;
            }
        }
    out[0] = sre; out[1] = sim; out[2] = sabs; out[3] = snb;
}

/* Brute force over all pairs and the 3x3 periodic images (global
 * coordinates), same definition; psi[2*p + k] per disk p (nullable). */
void orc_bruteforce_psi6(const double *xy, int64_t N, double Lx, double Ly, double rcut, double out[4], double *psi)
{
    const double rc2 = rcut * rcut;
    double sre = 0.0, sim = 0.0, sabs = 0.0, snb = 0.0;
    for (int64_t p = 0; p < N; ++p) {
        double are = 0.0, aim = 0.0;
        int nb = 0;
        for (int64_t q = 0; q < N; ++q)
            for (int iy = -1; iy <= 1; ++iy)
                for (int ix = -1; ix <= 1; ++ix) {
                    if (q == p && ix == 0 && iy == 0) continue;
                    double ddx = xy[2 * p] - (xy[2 * q] + ix * Lx), ddy = xy[2 * p + 1] - (xy[2 * q + 1] + iy * Ly);
                    double r2 = ddx * ddx + ddy * ddy;
                    if (!(r2 < rc2)) continue;
                    double ar = ddx * ddx - ddy * ddy, ai = 2.0 * (ddx * ddy);
                    double br = ar * ddx - ai * ddy, bi = ar * ddy + ai * ddx;
                    double cr = br * br - bi * bi, ci = 2.0 * (br * bi);
                    double r6 = (r2 * r2) * r2;
                    are += cr / r6;
                    aim += ci / r6;
                    nb += 1;
                }
        double pr = 0.0, pi = 0.0;
        if (nb > 0) { pr = are / (double)nb; pi = aim / (double)nb; }
        sre += pr; sim += pi; sabs += sqrt(pr * pr + pi * pi); snb += (double)nb;
        if (psi) { psi[2 * p] = pr; psi[2 * p + 1] = pi; }
    }
    out[0] = sre; out[1] = sim; out[2] = sabs; out[3] = snb;
}

/* ------------------------------------------------------------------------ */
/* Brute-force checks on global coordinates (tests)                          */
/* ------------------------------------------------------------------------ */
static double min_image(double d, double L)
{
    return d - L * floor(d / L + 0.5);
}

/* #unordered pairs with minimum-image distance < rmin. */
int64_t orc_bruteforce_close_pairs(const double *xy, int64_t N, double Lx, double Ly, double rmin)
{
    int64_t bad = 0;
    double r2min = rmin * rmin;
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = i + 1; j < N; ++j) {
            double dx = min_image(xy[2 * i] - xy[2 * j], Lx);
            double dy = min_image(xy[2 * i + 1] - xy[2 * j + 1], Ly);
            if (dx * dx + dy * dy < r2min) bad++;
        }
    return bad;
}

/* Ordered-pair distance histogram by brute force over all pairs and the 3x3
 * periodic images (global coordinates), same binning rule as above. */
void orc_bruteforce_histogram(const double *xy, int64_t N, double Lx, double Ly, double sigma,
                              int nbins, double dr, uint64_t *hist)
{
    memset(hist, 0, sizeof(uint64_t) * (size_t)nbins);
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < N; ++j) {
            for (int iy = -1; iy <= 1; ++iy)
                for (int ix = -1; ix <= 1; ++ix) {
                    if (i == j && ix == 0 && iy == 0) continue;
                    double dx = xy[2 * i] - (xy[2 * j] + (double)ix * Lx);
                    double dy = xy[2 * i + 1] - (xy[2 * j + 1] + (double)iy * Ly);
                    int b = bin_of_r2(dx * dx + dy * dy, sigma, dr, nbins);
                    if (b >= 0) hist[b] += 1;
                }
        }
}

int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int orc_local_overlaps(const oracle_t *o) { return (int)count_overlaps_local(o); }

/* ======================================================================== */
/* Three dimensions: N hard spheres of diameter sigma in a periodic          */
/* Lx x Ly x Lz box.  The method is the same with cubic cells and eight      */
/* checkerboard sets Q = (cx mod 2) + 2 (cy mod 2) + 4 (cz mod 2) (Sec. 2.1, */
/* Sec. 2.2: eight sub-sweeps per sweep in three dimensions; Sec. 6).       */
/* Readings (the paper gives the 3-d case in words only):                   */
/*  - grid: m_a = largest even integer <= L_a/sigma per axis (>= 4), and     */
/*    wx^2 + wy^2 + wz^2 < 4 sigma^2, so that each of the cell's eight half- */
/*    size boxes holds at most one centre: n <= 8 per cell;                 */
/*  - trial displacement uniform in a ball of radius d (the "maximum move    */
/*    radius" of Sec. 3.3), by rejection from (-1,1)^3;                     */
/*  - the shift direction is one of +-x, +-y, +-z (Alg. 4 with three axes); */
/*  - binary32 mode: directions from 21-bit fields as in two dimensions   */
/*    (three fields per attempt, two attempts per Philox block); positions, */
/*    widths and pair tests in binary32 (trial position and overlap         */
/*    predicate by fma).                                                    */
/* ======================================================================== */
#define NMAX3 8

typedef struct oracle3 {
    int64_t N;
    double L[3], sigma, d;
    int nsel;
    uint64_t seed;
    int prec;
    int m[3];
    double w[3];            /* cell widths, binary64 */
    float wf[3];            /* binary32 cell widths (FP32 mode) */
    int64_t C;              /* mx*my*mz */
    double *P;              /* FP64: coordinate a of slot (c,j) at P[3(8c+j)+a], c = (cz my + cy) mx + cx */
    float *Pf;              /* FP32 */
    uint8_t *n;
    double O[3];            /* accumulated grid origin */
    uint64_t sweep, shifts;
    uint64_t cnt[4];        /* trials, accepted, rejected (left cell), rejected (overlap) */
    int shuffle_particles, shuffle_sets;
} oracle3_t;

static const uint32_t kFactorial8[9] = {1u, 1u, 2u, 6u, 24u, 120u, 720u, 5040u, 40320u};

/* Fisher-Yates decode of k in [0, n!) for n <= 8 (same rule as decode_perm). */
static void decode_perm8(int n, uint32_t k, int perm[8])
{
    for (int j = 0; j < 8; ++j) perm[j] = j;
    for (int j = n - 1; j >= 1; --j) {
        int r = (int)(k % (uint32_t)(j + 1));
        k /= (uint32_t)(j + 1);
        int t = perm[j]; perm[j] = perm[r]; perm[r] = t;
    }
}

void orc3_decode_perm(int n, uint32_t k, int32_t out[8])
{
    int p[8];
    decode_perm8(n, k, p);
    for (int j = 0; j < 8; ++j) out[j] = p[j];
}

int orc3_grid(const double L[3], double sigma, int32_t m[3], double w[3])
{
    if (!(sigma > 0)) return ORC_EINVAL;
    for (int a = 0; a < 3; ++a) {
        if (!(L[a] > 0)) return ORC_EINVAL;
        int q = grid_size(L[a], sigma);
        if (q < 4) return ORC_EINVAL;
        m[a] = q;
        w[a] = L[a] / q;
    }
    if ((int64_t)m[0] * m[1] * m[2] >= ((int64_t)1 << 32)) return ORC_EINVAL;
    if (!((w[0] * w[0] + w[1] * w[1]) + w[2] * w[2] < 4.0 * sigma * sigma)) return ORC_EINVAL;
    return ORC_OK;
}

void orc3_destroy(oracle3_t *o)
{
    if (!o) return;
    free(o->P); free(o->Pf); free(o->n);
    free(o);
}

static oracle3_t *alloc_state3(int64_t N, const double L[3], double sigma, double d, int nsel,
                               uint64_t seed, int prec, int *err)
{
    int32_t m[3];
    double w[3];
    *err = ORC_EINVAL;
    if (N < 1 || nsel < 1 || nsel > 255 || (prec != 0 && prec != 1)) return NULL;
    if (orc3_grid(L, sigma, m, w) != ORC_OK) return NULL;
    for (int a = 0; a < 3; ++a)
        if (!(d > 0) || !(d < 0.5 * w[a])) return NULL;
    int64_t C = (int64_t)m[0] * m[1] * m[2];
    if (C * NMAX3 < N) return NULL;
    oracle3_t *o = (oracle3_t *)calloc(1, sizeof(oracle3_t));
    *err = ORC_ENOMEM;
    if (!o) return NULL;
    o->N = N; o->sigma = sigma; o->d = d; o->nsel = nsel; o->seed = seed; o->prec = prec;
    for (int a = 0; a < 3; ++a) { o->L[a] = L[a]; o->m[a] = m[a]; o->w[a] = w[a]; o->wf[a] = (float)w[a]; }
    o->C = C;
    o->shuffle_particles = 1; o->shuffle_sets = 1;
    o->n = (uint8_t *)calloc((size_t)C, 1);
    if (prec == 0) o->P = (double *)malloc(sizeof(double) * 3 * NMAX3 * (size_t)C);
    else o->Pf = (float *)malloc(sizeof(float) * 3 * NMAX3 * (size_t)C);
    if (!o->n || (prec == 0 ? !o->P : !o->Pf)) { orc3_destroy(o); return NULL; }
    *err = ORC_OK;
    return o;
}

static int64_t cell3(const oracle3_t *o, int cx, int cy, int cz)
{
    return ((int64_t)cz * o->m[1] + cy) * o->m[0] + cx;
}

static double slot3(const oracle3_t *o, int64_t c, int j, int a)
{
    return o->prec == 0 ? o->P[3 * (NMAX3 * c + j) + a] : (double)o->Pf[3 * (NMAX3 * c + j) + a];
}

/* binary32 overlap predicate in three dimensions:
 * fma(dx, dx, fma(dy, dy, fma(dz, dz, -sigma^2))) < 0. */
static int overlap3_32(float dx, float dy, float dz, float sig2)
{
    return fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, -sig2))) < 0.0f;
}

/* binary64 overlap predicate: (dx*dx + dy*dy) + dz*dz < sigma^2. */
static int overlap3_64(double dx, double dy, double dz, double sig2)
{
    return (dx * dx + dy * dy) + dz * dz < sig2;
}

/* Ordered overlapping pairs over each sphere's 27-cell neighbourhood, in
 * cell-local frames with the sweep's arithmetic. */
static int64_t count_overlaps_local3(const oracle3_t *o)
{
    int64_t bad = 0;
    for (int cz = 0; cz < o->m[2]; ++cz)
        for (int cy = 0; cy < o->m[1]; ++cy)
            for (int cx = 0; cx < o->m[0]; ++cx) {
                int64_t c = cell3(o, cx, cy, cz);
                for (int i = 0; i < o->n[c]; ++i)
                    for (int dz = -1; dz <= 1; ++dz)
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx) {
                                int64_t nc = cell3(o, (cx + dx + o->m[0]) % o->m[0], (cy + dy + o->m[1]) % o->m[1],
                                                   (cz + dz + o->m[2]) % o->m[2]);
                                for (int j = 0; j < o->n[nc]; ++j) {
                                    if (dx == 0 && dy == 0 && dz == 0 && j == i) continue;
                                    if (o->prec == 0) {
                                        double e0 = slot3(o, nc, j, 0) + (double)dx * o->w[0];
                                        double e1 = slot3(o, nc, j, 1) + (double)dy * o->w[1];
                                        double e2 = slot3(o, nc, j, 2) + (double)dz * o->w[2];
                                        if (overlap3_64(slot3(o, c, i, 0) - e0, slot3(o, c, i, 1) - e1,
                                                        slot3(o, c, i, 2) - e2, o->sigma * o->sigma))
                                            bad++;
                                    } else {
                                        float e0 = (float)slot3(o, nc, j, 0) + (float)dx * o->wf[0];
                                        float e1 = (float)slot3(o, nc, j, 1) + (float)dy * o->wf[1];
                                        float e2 = (float)slot3(o, nc, j, 2) + (float)dz * o->wf[2];
                                        if (overlap3_32((float)slot3(o, c, i, 0) - e0, (float)slot3(o, c, i, 1) - e1,
                                                        (float)slot3(o, c, i, 2) - e2,
                                                        (float)(o->sigma * o->sigma)))
                                            bad++;
                                    }
                                }
                            }
            }
    return bad;
}

/* Place global positions xyz[3N] into the cells (slot order = particle
 * order), with the same binning rule as in two dimensions. */
static int place3(oracle3_t *o, const double *xyz)
{
    memset(o->n, 0, (size_t)o->C);
    for (int64_t k = 0; k < 3 * NMAX3 * o->C; ++k) {
        if (o->prec == 0) o->P[k] = EMPTY_SLOT;
        else o->Pf[k] = (float)EMPTY_SLOT;
    }
    for (int64_t p = 0; p < o->N; ++p) {
        int cc[3];
        double l[3];
        for (int a = 0; a < 3; ++a) {
            double x = xyz[3 * p + a];
            if (!(x >= 0.0 && x <= o->L[a])) return ORC_EINVAL;
            bin_axis(x, o->w[a], o->m[a], &cc[a], &l[a]);
        }
        int64_t c = cell3(o, cc[0], cc[1], cc[2]);
        if (o->n[c] >= NMAX3) return ORC_EOVERFLOW;
        int j = o->n[c]++;
        for (int a = 0; a < 3; ++a) {
            if (o->prec == 0) o->P[3 * (NMAX3 * c + j) + a] = l[a];
            else {
                float f = (float)l[a];
                if (f >= o->wf[a]) f = prev_float(o->wf[a]);
                o->Pf[3 * (NMAX3 * c + j) + a] = f;
            }
        }
    }
    if (count_overlaps_local3(o) != 0) return ORC_EOVERLAP;
    return ORC_OK;
}

/* Face-centred cubic start: N = 4 q^3; unit cell b = (i,j,k) of side L_a/q
 * along axis a holds the sites (b + s + 1/4) L_a/q for the four basis
 * vectors s = (0,0,0), (1/2,1/2,0), (1/2,0,1/2), (0,1/2,1/2); site
 * p = 4((k q + j) q + i) + s is displaced uniformly within a ball of radius
 * 0.01 sigma (init stream of p, attempts of six words, binary64) and
 * wrapped into the box. */
int orc3_lattice_positions(int64_t N, const double L[3], double sigma, uint64_t seed, double *xyz)
{
    int64_t q = 1;
    while (4 * q * q * q < N) ++q;
    if (N < 4 || 4 * q * q * q != N) return ORC_EINVAL;
    static const double basis[4][3] = {{0, 0, 0}, {0.5, 0.5, 0}, {0.5, 0, 0.5}, {0, 0.5, 0.5}};
    const double rj = 0.01 * sigma;
    for (int64_t k = 0; k < q; ++k)
        for (int64_t j = 0; j < q; ++j)
            for (int64_t i = 0; i < q; ++i)
                for (int s = 0; s < 4; ++s) {
                    int64_t p = 4 * ((k * q + j) * q + i) + s;
                    const int64_t b[3] = {i, j, k};
                    stream_t st;
                    stream_open(&st, seed, (uint32_t)p, 0xFFFFFFFEu, DOM_INIT << 28);
                    double u[3];
                    do {
                        for (int a = 0; a < 3; ++a) {
                            uint32_t hi = stream_word(&st), lo = stream_word(&st);
                            u[a] = sym52(hi, lo);
                        }
                    } while (!((u[0] * u[0] + u[1] * u[1]) + u[2] * u[2] < 1.0));
                    for (int a = 0; a < 3; ++a) {
                        double x = ((double)b[a] + basis[s][a] + 0.25) * (L[a] / (double)q) + rj * u[a];
                        if (x >= L[a]) x -= L[a];
                        if (x < 0.0) x += L[a];
                        xyz[3 * p + a] = x;
                    }
                }
    return ORC_OK;
}

int orc3_create(oracle3_t **out, int64_t N, const double L[3], double sigma, double d, int nsel,
                uint64_t seed, int prec, const double *xyz)
{
    int err;
    *out = NULL;
    oracle3_t *o = alloc_state3(N, L, sigma, d, nsel, seed, prec, &err);
    if (!o) return err;
    if (xyz) {
        err = place3(o, xyz);
    } else {
        double *buf = (double *)malloc(sizeof(double) * 3 * (size_t)N);
        if (!buf) { orc3_destroy(o); return ORC_ENOMEM; }
        err = orc3_lattice_positions(N, L, sigma, seed, buf);
        if (err == ORC_OK) err = place3(o, buf);
        free(buf);
    }
    if (err != ORC_OK) { orc3_destroy(o); return err; }
    *out = o;
    return ORC_OK;
}

int orc3_set_move_size(oracle3_t *o, double d)
{
    for (int a = 0; a < 3; ++a)
        if (!(d > 0) || !(d < 0.5 * o->w[a])) return ORC_EINVAL;
    o->d = d;
    return ORC_OK;
}

void orc3_set_balance(oracle3_t *o, int shuffle_particles, int shuffle_sets)
{
    o->shuffle_particles = shuffle_particles;
    o->shuffle_sets = shuffle_sets;
}

/* Sweep-level draws: order of the eight sets by Fisher-Yates (j = 7..1,
 * k = bounded(j+1)), direction f = bounded(6) (f>>1 the axis, f&1 set for
 * the negative direction), distance unif53 * w_axis/2.  Explicit shifts draw
 * f and the distance from their own stream. */
typedef struct { int perm[8]; int fdir; double ds; } draws3_t;

static void sweep_draws3(uint64_t seed, uint32_t sweep, const double w[3], draws3_t *r)
{
    stream_t s;
    stream_open(&s, seed, sweep, 0xFFFFFFFFu, DOM_SWEEP << 28);
    for (int q = 0; q < 8; ++q) r->perm[q] = q;
    for (int j = 7; j >= 1; --j) {
        int k = (int)stream_bounded(&s, (uint32_t)(j + 1));
        int t = r->perm[j]; r->perm[j] = r->perm[k]; r->perm[k] = t;
    }
    r->fdir = (int)stream_bounded(&s, 6u);
    uint32_t hi = stream_word(&s), lo = stream_word(&s);
    r->ds = unif53(hi, lo) * (0.5 * w[r->fdir >> 1]);
}

static void shift_draws3(uint64_t seed, uint32_t index, const double w[3], draws3_t *r)
{
    stream_t s;
    stream_open(&s, seed, index, 0xFFFFFFFFu, DOM_SHIFT << 28);
    for (int q = 0; q < 8; ++q) r->perm[q] = q;
    r->fdir = (int)stream_bounded(&s, 6u);
    uint32_t hi = stream_word(&s), lo = stream_word(&s);
    r->ds = unif53(hi, lo) * (0.5 * w[r->fdir >> 1]);
}

void orc3_sweep_draws(uint64_t seed, uint32_t sweep, const double w[3], int32_t perm[8], int32_t *fdir, double *ds)
{
    draws3_t r;
    sweep_draws3(seed, sweep, w, &r);
    for (int q = 0; q < 8; ++q) perm[q] = r.perm[q];
    *fdir = r.fdir;
    *ds = r.ds;
}

/* Draws of one cell update (sweep s, set Q, canonical cell c): shuffle
 * stream S = (s, c, (0<<28)|(Q<<24)) gives k = bounded(n!) when n >= 2 and
 * the particle shuffle is on (both modes); trial stream
 * T = (s, c, (1<<28)|(Q<<24)) gives the directions, uniform in the unit ball
 * by rejection from (-1,1)^3:
 *   binary64: consecutive words, six per attempt: u = sym52(w0,w1),
 *             v = sym52(w2,w3), s = sym52(w4,w5), kept when
 *             (u*u + v*v) + s*s < 1;
 *   binary32: block b cut into six 21-bit fields; attempts are the field
 *             triples (0,1,2), (3,4,5) of blocks 0, 1, ...: u = sym21,
 *             kept when fma(u, u, fma(v, v, s*s)) < 1 in binary32. */
static void cell_draws3(uint64_t seed, uint32_t sweep, uint32_t cell, int Q, int n, int shuffle, int nsel,
                        int prec, int perm[8], double *U)
{
    const uint32_t setbits = (uint32_t)Q << 24;
    for (int j = 0; j < 8; ++j) perm[j] = j;
    if (shuffle && n >= 2) {
        stream_t s;
        stream_open(&s, seed, sweep, cell, (DOM_SHUFFLE << 28) | setbits);
        decode_perm8(n, stream_bounded(&s, kFactorial8[n]), perm);
    }
    if (prec == 0) {
        stream_t t;
        stream_open(&t, seed, sweep, cell, (DOM_TRIAL << 28) | setbits);
        for (int k = 0; k < nsel;) {
            double u[3];
            for (int a = 0; a < 3; ++a) {
                uint32_t hi = stream_word(&t), lo = stream_word(&t);
                u[a] = sym52(hi, lo);
            }
            if ((u[0] * u[0] + u[1] * u[1]) + u[2] * u[2] < 1.0) {
                U[3 * k] = u[0]; U[3 * k + 1] = u[1]; U[3 * k + 2] = u[2];
                ++k;
            }
        }
    } else {
        uint32_t block = 0, w[4], f[6];
        int triple = 2;
        for (int k = 0; k < nsel;) {
            if (triple == 2) {
                philox_block(seed, sweep, cell, (DOM_TRIAL << 28) | setbits, block++, w);
                fields21(w, f);
                triple = 0;
            }
            float u = sym21(f[3 * triple]), v = sym21(f[3 * triple + 1]), t = sym21(f[3 * triple + 2]);
            ++triple;
            if (fmaf(u, u, fmaf(v, v, t * t)) < 1.0f) {
                U[3 * k] = u; U[3 * k + 1] = v; U[3 * k + 2] = t;
                ++k;
            }
        }
    }
}

/* Test hook: the draws of one cell update (perm[8], uvw[3*nsel]). */
void orc3_cell_draws(uint64_t seed, uint32_t sweep, uint32_t cell, int Q, int n, int shuffle, int nsel, int prec,
                     int32_t perm[8], double *uvw)
{
    int p[8];
    cell_draws3(seed, sweep, cell, Q, n, shuffle, nsel, prec, p, uvw);
    for (int j = 0; j < 8; ++j) perm[j] = p[j];
}

/* One cell update (Alg. 1, Alg. 2 in three dimensions). */
static void cell_update3(oracle3_t *o, uint32_t sweep, int Q, int cx, int cy, int cz, uint64_t acc[4])
{
    int64_t c = cell3(o, cx, cy, cz);
    int n = o->n[c];
    if (n == 0) return;
    int perm[8];
    double U[3 * 256];
    cell_draws3(o->seed, sweep, (uint32_t)c, Q, n, o->shuffle_particles, o->nsel, o->prec, perm, U);
    const int cc[3] = {cx, cy, cz};
    if (o->prec == 0) {
        double *X = o->P + 3 * NMAX3 * c;
        double tmp[3 * NMAX3];
        for (int j = 0; j < n; ++j)
            for (int a = 0; a < 3; ++a) tmp[3 * j + a] = X[3 * perm[j] + a];
        for (int j = 0; j < 3 * n; ++j) X[j] = tmp[j];
        const double sig2 = o->sigma * o->sigma;
        for (int t = 0; t < o->nsel; ++t) {
            int i = visit_slot(t, n);
            double p[3];
            int inside = 1;
            for (int a = 0; a < 3; ++a) {
                p[a] = X[3 * i + a] + o->d * U[3 * t + a];
                if (!(p[a] >= 0.0 && p[a] < o->w[a])) inside = 0;
            }
            acc[0]++;
            if (!inside) { acc[2]++; continue; }
            int overlap = 0;
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                if (overlap3_64(p[0] - X[3 * j], p[1] - X[3 * j + 1], p[2] - X[3 * j + 2], sig2)) overlap = 1;
            }
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (dx == 0 && dy == 0 && dz == 0) continue;
                        const int dd[3] = {dx, dy, dz};
                        int nn[3];
                        for (int a = 0; a < 3; ++a) nn[a] = (cc[a] + dd[a] + o->m[a]) % o->m[a];
                        int64_t nc = cell3(o, nn[0], nn[1], nn[2]);
                        const double *Y = o->P + 3 * NMAX3 * nc;
                        for (int j = 0; j < o->n[nc]; ++j) {
                            double e[3];
                            for (int a = 0; a < 3; ++a) e[a] = Y[3 * j + a] + (double)dd[a] * o->w[a];
                            if (overlap3_64(p[0] - e[0], p[1] - e[1], p[2] - e[2], sig2)) overlap = 1;
                        }
                    }
            if (overlap) { acc[3]++; continue; }
            for (int a = 0; a < 3; ++a) X[3 * i + a] = p[a];
            acc[1]++;
        }
    } else {
        float *X = o->Pf + 3 * NMAX3 * c;
        float tmp[3 * NMAX3];
        for (int j = 0; j < n; ++j)
            for (int a = 0; a < 3; ++a) tmp[3 * j + a] = X[3 * perm[j] + a];
        for (int j = 0; j < 3 * n; ++j) X[j] = tmp[j];
        const float sig2 = (float)(o->sigma * o->sigma);
        const float df = (float)o->d;
        for (int t = 0; t < o->nsel; ++t) {
            int i = visit_slot(t, n);
            float p[3];
            int inside = 1;
            for (int a = 0; a < 3; ++a) {
                p[a] = fmaf(df, (float)U[3 * t + a], X[3 * i + a]);   /* U exact in binary32 */
                if (!(p[a] >= 0.0f && p[a] < o->wf[a])) inside = 0;
            }
            acc[0]++;
            if (!inside) { acc[2]++; continue; }
            int overlap = 0;
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                if (overlap3_32(p[0] - X[3 * j], p[1] - X[3 * j + 1], p[2] - X[3 * j + 2], sig2)) overlap = 1;
            }
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (dx == 0 && dy == 0 && dz == 0) continue;
                        const int dd[3] = {dx, dy, dz};
                        int nn[3];
                        for (int a = 0; a < 3; ++a) nn[a] = (cc[a] + dd[a] + o->m[a]) % o->m[a];
                        int64_t nc = cell3(o, nn[0], nn[1], nn[2]);
                        const float *Y = o->Pf + 3 * NMAX3 * nc;
                        for (int j = 0; j < o->n[nc]; ++j) {
                            float e[3];
                            for (int a = 0; a < 3; ++a) e[a] = Y[3 * j + a] + (float)dd[a] * o->wf[a];
                            if (overlap3_32(p[0] - e[0], p[1] - e[1], p[2] - e[2], sig2)) overlap = 1;
                        }
                    }
            if (overlap) { acc[3]++; continue; }
            for (int a = 0; a < 3; ++a) X[3 * i + a] = p[a];
            acc[1]++;
        }
    }
}

/* All cells of set Q (independent of each other). */
static void subsweep3(oracle3_t *o, uint32_t sweep, int Q)
{
    int qx = Q & 1, qy = (Q >> 1) & 1, qz = Q >> 2;
    uint64_t t0 = 0, t1 = 0, t2 = 0, t3 = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(+ : t0, t1, t2, t3)
#endif
    for (int cz = qz; cz < o->m[2]; cz += 2) {
        uint64_t acc[4] = {0, 0, 0, 0};
        for (int cy = qy; cy < o->m[1]; cy += 2)
            for (int cx = qx; cx < o->m[0]; cx += 2) cell_update3(o, sweep, Q, cx, cy, cz, acc);
        t0 += acc[0]; t1 += acc[1]; t2 += acc[2]; t3 += acc[3];
    }
    o->cnt[0] += t0; o->cnt[1] += t1; o->cnt[2] += t2; o->cnt[3] += t3;
}

/* Cell shift (Alg. 4) along one of three axes, the same rule as in two
 * dimensions: new cell c keeps the spheres of old c that stay inside it, in
 * slot order, then takes those of old c+f that leave c+f, re-expressed in
 * c's frame and clamped into [0, w). */
static int shift_cells3(oracle3_t *o, int fdir, double ds)
{
    const int ax = fdir >> 1;
    const int sgn = (fdir & 1) ? -1 : 1;
    const int64_t C = o->C;
    uint8_t *nn = (uint8_t *)calloc((size_t)C, 1);
    double *NP = NULL;
    float *NPf = NULL;
    if (o->prec == 0) NP = (double *)malloc(sizeof(double) * 3 * NMAX3 * (size_t)C);
    else NPf = (float *)malloc(sizeof(float) * 3 * NMAX3 * (size_t)C);
    if (!nn || (o->prec == 0 ? !NP : !NPf)) { free(nn); free(NP); free(NPf); return ORC_ENOMEM; }
    int overflow = 0;
    for (int cz = 0; cz < o->m[2]; ++cz)
        for (int cy = 0; cy < o->m[1]; ++cy)
            for (int cx = 0; cx < o->m[0]; ++cx) {
                int64_t c = cell3(o, cx, cy, cz);
                int nb3[3] = {cx, cy, cz};
                nb3[ax] = (nb3[ax] + sgn + o->m[ax]) % o->m[ax];
                int64_t nb = cell3(o, nb3[0], nb3[1], nb3[2]);
                int k = 0;
                if (o->prec == 0) {
                    const double w = o->w[ax], sd = (double)sgn * ds, sw = (double)sgn * w;
                    double tmp[3 * (2 * NMAX3)];
                    for (int j = 0; j < o->n[c]; ++j) {
                        const double *p = o->P + 3 * (NMAX3 * c + j);
                        double dp = p[ax] - sd;
                        if (dp >= 0.0 && dp < w) {
                            for (int a = 0; a < 3; ++a) tmp[3 * k + a] = p[a];
                            tmp[3 * k + ax] = dp;
                            k++;
                        }
                    }
                    for (int j = 0; j < o->n[nb]; ++j) {
                        const double *p = o->P + 3 * (NMAX3 * nb + j);
                        double dp = p[ax] - sd;
                        if (!(dp >= 0.0 && dp < w)) {
                            double v = dp + sw;
                            if (v >= w) v = prev_double(w);
                            if (v < 0.0) v = 0.0;
                            for (int a = 0; a < 3; ++a) tmp[3 * k + a] = p[a];
                            tmp[3 * k + ax] = v;
                            k++;
                        }
                    }
                    if (k > NMAX3) { overflow = 1; k = NMAX3; }
                    for (int j = 0; j < 3 * NMAX3; ++j) NP[3 * NMAX3 * c + j] = j < 3 * k ? tmp[j] : EMPTY_SLOT;
                } else {
                    const float w = o->wf[ax], sd = (float)sgn * (float)ds, sw = (float)sgn * w;
                    float tmp[3 * (2 * NMAX3)];
                    for (int j = 0; j < o->n[c]; ++j) {
                        const float *p = o->Pf + 3 * (NMAX3 * c + j);
                        float dp = p[ax] - sd;
                        if (dp >= 0.0f && dp < w) {
                            for (int a = 0; a < 3; ++a) tmp[3 * k + a] = p[a];
                            tmp[3 * k + ax] = dp;
                            k++;
                        }
                    }
                    for (int j = 0; j < o->n[nb]; ++j) {
                        const float *p = o->Pf + 3 * (NMAX3 * nb + j);
                        float dp = p[ax] - sd;
                        if (!(dp >= 0.0f && dp < w)) {
                            float v = dp + sw;
                            if (v >= w) v = prev_float(w);
                            if (v < 0.0f) v = 0.0f;
                            for (int a = 0; a < 3; ++a) tmp[3 * k + a] = p[a];
                            tmp[3 * k + ax] = v;
                            k++;
                        }
                    }
                    if (k > NMAX3) { overflow = 1; k = NMAX3; }
                    for (int j = 0; j < 3 * NMAX3; ++j)
                        NPf[3 * NMAX3 * c + j] = j < 3 * k ? tmp[j] : (float)EMPTY_SLOT;
                }
                nn[c] = (uint8_t)k;
            }
    if (o->prec == 0) {
        free(o->P);
        o->P = NP;
        o->O[ax] += (double)sgn * ds;
    } else {
        free(o->Pf);
        o->Pf = NPf;
        o->O[ax] += (double)((float)sgn * (float)ds);
    }
    free(o->n);
    o->n = nn;
    return overflow ? ORC_EOVERFLOW : ORC_OK;
}

int orc3_sweep(oracle3_t *o, int64_t nsweeps)
{
    for (int64_t k = 0; k < nsweeps; ++k) {
        uint32_t sweep = (uint32_t)o->sweep;
        draws3_t r;
        sweep_draws3(o->seed, sweep, o->w, &r);
        for (int q = 0; q < 8; ++q) subsweep3(o, sweep, o->shuffle_sets ? r.perm[q] : q);
        int err = shift_cells3(o, r.fdir, r.ds);
        o->sweep += 1;
        if (err != ORC_OK) return err;
    }
    return ORC_OK;
}

int orc3_shift(oracle3_t *o)
{
    draws3_t r;
    shift_draws3(o->seed, (uint32_t)o->shifts, o->w, &r);
    o->shifts += 1;
    return shift_cells3(o, r.fdir, r.ds);
}

void orc3_subsweep(oracle3_t *o, uint32_t sweep, int Q) { subsweep3(o, sweep, Q); }

void orc3_info(const oracle3_t *o, int32_t m[3], double w[3], uint64_t *sweep, uint64_t *shifts)
{
    for (int a = 0; a < 3; ++a) { m[a] = o->m[a]; w[a] = o->w[a]; }
    *sweep = o->sweep;
    *shifts = o->shifts;
}

void orc3_counters(const oracle3_t *o, uint64_t out[4])
{
    for (int k = 0; k < 4; ++k) out[k] = o->cnt[k];
}

void orc3_origin(const oracle3_t *o, double out[3])
{
    for (int a = 0; a < 3; ++a) out[a] = o->O[a];
}

/* Raw state: local[3(8c+j)+a] (EMPTY_SLOT where unused), counts[c]. */
void orc3_state(const oracle3_t *o, double *local, uint8_t *counts)
{
    for (int64_t c = 0; c < o->C; ++c) {
        counts[c] = o->n[c];
        for (int j = 0; j < NMAX3; ++j)
            for (int a = 0; a < 3; ++a)
                local[3 * (NMAX3 * c + j) + a] = j < o->n[c] ? slot3(o, c, j, a) : EMPTY_SLOT;
    }
}

/* Global coordinates in canonical (cell, slot) order:
 * g = O + (cell*w + local) wrapped into [0, m*w) (binary32 widths in FP32 mode). */
void orc3_positions(const oracle3_t *o, double *xyz)
{
    double w[3], L[3];
    for (int a = 0; a < 3; ++a) {
        w[a] = o->prec == 0 ? o->w[a] : (double)o->wf[a];
        L[a] = o->prec == 0 ? o->L[a] : (double)o->m[a] * w[a];
    }
    int64_t p = 0;
    for (int cz = 0; cz < o->m[2]; ++cz)
        for (int cy = 0; cy < o->m[1]; ++cy)
            for (int cx = 0; cx < o->m[0]; ++cx) {
                int64_t c = cell3(o, cx, cy, cz);
                const int cc[3] = {cx, cy, cz};
                for (int j = 0; j < o->n[c]; ++j) {
                    for (int a = 0; a < 3; ++a) {
                        double g = o->O[a] + ((double)cc[a] * w[a] + slot3(o, c, j, a));
                        xyz[3 * p + a] = g - L[a] * floor(g / L[a]);
                    }
                    p++;
                }
            }
}

/* Contact histogram in three dimensions: ordered pairs at distance r with
 * sigma <= r < sigma + nbins*dr over the 5x5x5 cell neighbourhood, binary64,
 * squared distance (dx*dx + dy*dy) + dz*dz, bins as in two dimensions. */
void orc3_histogram(const oracle3_t *o, int nbins, double dr, uint64_t *hist)
{
    memset(hist, 0, sizeof(uint64_t) * (size_t)nbins);
    double w[3];
    for (int a = 0; a < 3; ++a) w[a] = o->prec == 0 ? o->w[a] : (double)o->wf[a];
    for (int cz = 0; cz < o->m[2]; ++cz)
        for (int cy = 0; cy < o->m[1]; ++cy)
            for (int cx = 0; cx < o->m[0]; ++cx) {
                int64_t c = cell3(o, cx, cy, cz);
                const int cc[3] = {cx, cy, cz};
                for (int i = 0; i < o->n[c]; ++i)
                    for (int dz = -2; dz <= 2; ++dz)
                        for (int dy = -2; dy <= 2; ++dy)
                            for (int dx = -2; dx <= 2; ++dx) {
                                const int dd[3] = {dx, dy, dz};
                                int nn[3];
                                for (int a = 0; a < 3; ++a) nn[a] = ((cc[a] + dd[a]) % o->m[a] + o->m[a]) % o->m[a];
                                int64_t nc = cell3(o, nn[0], nn[1], nn[2]);
                                for (int j = 0; j < o->n[nc]; ++j) {
                                    if (dx == 0 && dy == 0 && dz == 0 && j == i) continue;
                                    double e[3];
                                    for (int a = 0; a < 3; ++a)
                                        e[a] = slot3(o, c, i, a) - (slot3(o, nc, j, a) + (double)dd[a] * w[a]);
                                    int b = bin_of_r2((e[0] * e[0] + e[1] * e[1]) + e[2] * e[2], o->sigma, dr, nbins);
                                    if (b >= 0) hist[b] += 1;
                                }
                            }
            }
}

int orc3_local_overlaps(const oracle3_t *o) { return (int)count_overlaps_local3(o); }

/* Brute force on global coordinates over all pairs and the 27 periodic
 * images (tests): unordered pairs closer than rmin, and the ordered-pair
 * distance histogram with the rule above. */
int64_t orc3_bruteforce_close_pairs(const double *xyz, int64_t N, const double L[3], double rmin)
{
    int64_t bad = 0;
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = i + 1; j < N; ++j) {
            double e[3];
            for (int a = 0; a < 3; ++a) e[a] = min_image(xyz[3 * i + a] - xyz[3 * j + a], L[a]);
            if ((e[0] * e[0] + e[1] * e[1]) + e[2] * e[2] < rmin * rmin) bad++;
        }
    return bad;
}

void orc3_bruteforce_histogram(const double *xyz, int64_t N, const double L[3], double sigma, int nbins,
                               double dr, uint64_t *hist)
{
    memset(hist, 0, sizeof(uint64_t) * (size_t)nbins);
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < N; ++j)
            for (int iz = -1; iz <= 1; ++iz)
                for (int iy = -1; iy <= 1; ++iy)
                    for (int ix = -1; ix <= 1; ++ix) {
                        if (i == j && ix == 0 && iy == 0 && iz == 0) continue;
                        const int ii[3] = {ix, iy, iz};
                        double e[3];
                        for (int a = 0; a < 3; ++a) e[a] = xyz[3 * i + a] - (xyz[3 * j + a] + (double)ii[a] * L[a]);
                        int b = bin_of_r2((e[0] * e[0] + e[1] * e[1]) + e[2] * e[2], sigma, dr, nbins);
                        if (b >= 0) hist[b] += 1;
                    }
}
