/*
 * fic_oracle.c -- plain CPU oracle for the modified fast fractal encoder of
 * Salarian & Miar Naimi, "Modified Fast Fractal Image Compression Algorithm in
 * spatial domain" (arXiv 1502.00324).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may load this
 * library: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py do.  It shares no code, header, table or helper
 * with the CUDA path; the two meet only in the seeded input images.
 *
 * Every step is written as a plain loop in the paper's order:
 *   Sec. 2    ranges: non-overlapping BxB blocks, left->right, top->bottom;
 *             domains: all 2Bx2B blocks at integer step L, decimated 2x2;
 *             the eight isometries (rotations by 0/90/180/270 degrees
 *             clockwise, and each one mirrored).
 *   Eq. 1     E(R,D) = sum_i (S d_i + O - r_i)^2.
 *   Eq. 3     O = mean(R) - S mean(D)   (least-squares optimal offset).
 *   Eq. 5-6   block entropy from grey-level counts (here in bits).
 *   Sec. 3    domain pool = domains with entropy greater than a threshold;
 *   Sec. 4    or the DN domains of highest entropy (the experiments' pools).
 *   Sec. 3.2  predefined contrast factors S per step instead of a search.
 *   Sec. 2    quadtree steps: a range whose error exceeds the step threshold
 *             splits into four; the last step stores its best mapping anyway.
 *   Sec. 3.3  stored record: step, range mean, isometry, domain address, S.
 *   Eq. 4     PSNR.
 *
 * Readings of points the paper leaves open:
 *   - decimation is the 2x2 average, carried as the integer 2x2 SUM d' so
 *     that d = d'/4 and all arithmetic stays integral;
 *   - S = p/q with one common denominator q per step;
 *   - selection and the split test use the exact error at the optimal
 *     (unquantised) offset: the integer score 16 q^2 n E(S, O*) with
 *     n = B*B, written out below;
 *   - ties go to the lowest (pool index, isometry, S index);
 *   - the split test is "RMS error > tol" with tol quantised to 1/16 grey
 *     level (e16 = round(16 tol));
 *   - the stored offset is the range mean quantised to 7 bits,
 *     o_q = min(127, floor(sum(r) / (2n))), decoded as 2 o_q + 1;
 *   - entropy is summed in ascending order of the grey-level counts, so
 *     equal count multisets give identical values; the top-DN pool compares
 *     entropies rounded to 2^-20 bit and takes equal ones in raster order;
 *   - entropy threshold < 0 admits every domain; an empty pool at a
 *     non-final step splits every range, at the final step it stores a
 *     mean-only record (pool index 0xFFFFFFFF);
 *   - decoding starts from a constant 128 image and applies all mappings to
 *     the previous iterate (Jacobi) until a fixed point or a cap.
 *
 * Parity status: every function here is pinned by tests that do not use
 * the oracle's own formulas (tests/test_oracle_pins.py: brute force, exact
 * rationals, closed forms, library routines, the paper's printed counts);
 * the pins are themselves checked by planting mistakes in copies of this
 * file (tests/test_oracle_mutations.py).  Parity unpinned: the absolute
 * quality of an encode (PSNR, compression ratio) against the paper's
 * tables, whose test images are not available.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Records and options (layouts private to the oracle).                */
/* ------------------------------------------------------------------ */

/* One stored record per coded range (Sec. 3.3, Fig. 7).  Positions are kept
 * explicitly for checking; score is the exact 16 q^2 n E of the mapping. */
typedef struct {
    int32_t rx, ry;       /* range top-left, pixels                       */
    int32_t level;        /* quadtree step, 0 = largest block            */
    int32_t B;            /* range side                                   */
    int32_t iso;          /* isometry index 0..7                          */
    int32_t s_idx;        /* index into the step's S set, -1: mean only   */
    int32_t o_q;          /* 7-bit range mean                             */
    int32_t dx, dy;       /* domain top-left, pixels                      */
    uint32_t pool_idx;    /* address in the step's domain list           */
    int64_t score;        /* 16 q^2 n E at the optimal offset             */
} or_code;

#define OR_MAX_S 16
#define OR_MAX_LEVELS 5

typedef struct {
    int n_s;              /* number of contrast factors at this step      */
    int q;                /* common denominator                           */
    int p[OR_MAX_S];      /* S_i = p[i] / q                               */
} or_sset;

/* A step's domain pool: the admitted 2Bx2B positions in raster order and
 * their decimated blocks (B x B sums of 2x2 pixels). */
typedef struct {
    int B, L, n_pos;           /* side, step, number of candidate positions */
    int64_t dn;                /* admitted count (pool size DN)              */
    int32_t* x;                /* admitted positions, raster order           */
    int32_t* y;
    int32_t* dsum;             /* decimated block: dn * B * B values         */
    int64_t* sum_d;            /* sum of d' over the block                  */
    int64_t* sum_d2;           /* sum of d'^2 over the block                */
    int64_t near_thresh;       /* positions with |H - thr| < 1e-9           */
} or_pool;

/* ------------------------------------------------------------------ */
/* Sec. 2: the eight isometries on a B x B block, out[i][j] (row, col).  */
/* ------------------------------------------------------------------ */

/* rot: 90 degrees clockwise, out[i][j] = in[B-1-j][i]. */
static void rot90cw(const int32_t* in, int B, int32_t* out)
{
    for (int i = 0; i < B; ++i)
        for (int j = 0; j < B; ++j)
            out[i * B + j] = in[(B - 1 - j) * B + i];
}

/* mirror: out[i][j] = in[i][B-1-j]. */
static void mirror(const int32_t* in, int B, int32_t* out)
{
    for (int i = 0; i < B; ++i)
        for (int j = 0; j < B; ++j)
            out[i * B + j] = in[i * B + (B - 1 - j)];
}

/* T_k = rot^k for k < 4 and mirror(rot^(k-4)) for k >= 4.  B <= 32. */
void or_isometry(const int32_t* in, int B, int k, int32_t* out)
{
    int32_t a[32 * 32], b[32 * 32];
    int n = B * B;
    memcpy(a, in, sizeof(int32_t) * n);
    for (int r = 0; r < (k & 3); ++r) {
        rot90cw(a, B, b);
        memcpy(a, b, sizeof(int32_t) * n);
    }
    if (k >= 4) {
        mirror(a, B, b);
        memcpy(a, b, sizeof(int32_t) * n);
    }
    memcpy(out, a, sizeof(int32_t) * n);
}

/* ------------------------------------------------------------------ */
/* Sec. 2: decimated domain, B x B sums of 2x2 pixels of a 2B x 2B block. */
/* ------------------------------------------------------------------ */
void or_decimate(const uint8_t* img, int N, int x, int y, int B, int32_t* out)
{
    for (int i = 0; i < B; ++i)
        for (int j = 0; j < B; ++j) {
            int yy = y + 2 * i, xx = x + 2 * j;
            out[i * B + j] = (int32_t)img[yy * N + xx] + img[yy * N + xx + 1] +
                             img[(yy + 1) * N + xx] + img[(yy + 1) * N + xx + 1];
        }
}

/* ------------------------------------------------------------------ */
/* Eq. 5-6: entropy of the grey levels of a size x size block, in bits. */
/* p_i = q_i / (number of pixels); H = -sum_i p_i log2 p_i over levels  */
/* present, summed in ascending grey level.                            */
/* ------------------------------------------------------------------ */
double or_entropy_bits(const uint8_t* img, int N, int x, int y, int size)
{
    int64_t count[256];
    memset(count, 0, sizeof(count));
    for (int i = 0; i < size; ++i)
        for (int j = 0; j < size; ++j)
            count[img[(y + i) * N + x + j]] += 1;
    /* The non-zero counts in ascending order: the sum then depends only on
     * the multiset of counts, so blocks whose histograms are permutations
     * of each other (equal entropy) get bit-identical values. */
    int64_t c[256];
    int m = 0;
    for (int g = 0; g < 256; ++g) {
        if (count[g] == 0) continue;
        int k = m++;
        while (k > 0 && c[k - 1] > count[g]) { c[k] = c[k - 1]; --k; }
        c[k] = count[g];
    }
    double total = (double)size * (double)size;
    double h = 0.0;
    for (int k = 0; k < m; ++k) {
        double p = (double)c[k] / total;
        h -= p * log2(p);
    }
    return h;
}

/* ------------------------------------------------------------------ */
/* Exact error of one candidate mapping.                              */
/*                                                                    */
/* With d = d'/4, S = p/q and O at its optimum (eq. 3), eq. 1 becomes  */
/*   n E = Vr - 2 S (Crd/4) + S^2 (Vd/16),                             */
/* where Vr = n sum r^2 - (sum r)^2, Crd = n sum r d' - sum r sum d',  */
/* Vd = n sum d'^2 - (sum d')^2.  Multiplying by 16 q^2 gives the      */
/* integer score                                                       */
/*   16 q^2 n E = 16 q^2 Vr - 8 p q Crd + p^2 Vd.                      */
/* ------------------------------------------------------------------ */
static int64_t score_from_sums(int64_t n, int64_t sr, int64_t sr2, int64_t sd,
                               int64_t sd2, int64_t srd, int64_t p, int64_t q)
{
    int64_t vr = n * sr2 - sr * sr;
    int64_t crd = n * srd - sr * sd;
    int64_t vd = n * sd2 - sd * sd;
    return 16 * q * q * vr - 8 * p * q * crd + p * p * vd;
}

/* Score of range r (B x B grey levels) against decimated domain dsum under
 * isometry k and S = p/q: the domain is transformed by T_k and compared to
 * the range pixel by pixel. */
int64_t or_score(const int32_t* r, const int32_t* dsum, int B, int k, int p, int q)
{
    int32_t t[32 * 32];
    or_isometry(dsum, B, k, t);
    int64_t n = (int64_t)B * B, sr = 0, sr2 = 0, sd = 0, sd2 = 0, srd = 0;
    for (int i = 0; i < n; ++i) {
        sr += r[i];
        sr2 += (int64_t)r[i] * r[i];
        sd += t[i];
        sd2 += (int64_t)t[i] * t[i];
        srd += (int64_t)r[i] * t[i];
    }
    return score_from_sums(n, sr, sr2, sd, sd2, srd, p, q);
}

/* ------------------------------------------------------------------ */
/* Sec. 2 / Sec. 3: one step's domain pool.                           */
/* ------------------------------------------------------------------ */
void or_pool_free(or_pool* pl)
{
    free(pl->x); free(pl->y); free(pl->dsum); free(pl->sum_d); free(pl->sum_d2);
    memset(pl, 0, sizeof(*pl));
}

/* Number of domain positions along one axis: x = 0, L, 2L, ... <= N - 2B. */
int or_positions_per_axis(int N, int B, int L)
{
    if (N < 2 * B) return 0;
    return (N - 2 * B) / L + 1;
}

/* Top-DN ranking key: entropy rounded to a multiple of 2^-20 bit (half
 * up), larger first; equal rounded entropies in raster order.  Rounding to
 * nearest keeps the many exactly dyadic entropies (all counts powers of
 * two) at the centre of their step, far from any rounding boundary. */
typedef struct { int64_t hq; int64_t i; } or_rank;

#define OR_HQ_SCALE 1048576.0  /* 2^20 */

static int cmp_rank(const void* a, const void* b)
{
    const or_rank* u = (const or_rank*)a;
    const or_rank* v = (const or_rank*)b;
    if (u->hq != v->hq) return u->hq > v->hq ? -1 : 1;
    return (u->i > v->i) - (u->i < v->i);
}

/* Pool rules (Sec. 3, Sec. 3.2.1, Sec. 4):
 *   dn_top <= 0: every position whose entropy is greater than thr (thr < 0
 *                admits all);
 *   dn_top > 0:  the dn_top positions of highest entropy ("we choose blocks
 *                with the highest entropy"), entropies compared at 2^-20 bit
 *                (floor(H 2^20 + 1/2)), equal ones taken in raster order;
 *                near_thresh then counts positions of the boundary value
 *                (+-1) whose H 2^20 + 1/2 lies within 1e-6 of an integer,
 *                where rounding could move them across a step.
 * Either way the admitted positions are listed in raster order and the list
 * index is the domain address (Sec. 3.3). */
int or_pool_build_ex(const uint8_t* img, int N, int B, int L, double thr, int64_t dn_top,
                     or_pool* pl)
{
    memset(pl, 0, sizeof(*pl));
    int per = or_positions_per_axis(N, B, L);
    int n = B * B;
    pl->B = B; pl->L = L; pl->n_pos = per * per;
    pl->x = (int32_t*)malloc(sizeof(int32_t) * (size_t)(pl->n_pos ? pl->n_pos : 1));
    pl->y = (int32_t*)malloc(sizeof(int32_t) * (size_t)(pl->n_pos ? pl->n_pos : 1));
    if (!pl->x || !pl->y) return -1;
    char* admit = (char*)calloc((size_t)(pl->n_pos ? pl->n_pos : 1), 1);
    if (!admit) return -1;
    if (dn_top > 0) {
        or_rank* r = (or_rank*)malloc(sizeof(or_rank) * (size_t)(pl->n_pos ? pl->n_pos : 1));
        if (!r) { free(admit); return -1; }
        double* hx = (double*)malloc(sizeof(double) * (size_t)(pl->n_pos ? pl->n_pos : 1));
        if (!hx) { free(r); free(admit); return -1; }
        for (int64_t i = 0; i < pl->n_pos; ++i) {
            double h = or_entropy_bits(img, N, (int)(i % per) * L, (int)(i / per) * L, 2 * B);
            hx[i] = h * OR_HQ_SCALE + 0.5;
            r[i].hq = (int64_t)floor(hx[i]);
            r[i].i = i;
        }
        qsort(r, (size_t)pl->n_pos, sizeof(or_rank), cmp_rank);
        int64_t take = dn_top < pl->n_pos ? dn_top : pl->n_pos;
        for (int64_t k = 0; k < take; ++k) admit[r[k].i] = 1;
        if (take > 0 && take < pl->n_pos) {
            int64_t hb = r[take - 1].hq;
            for (int64_t i = 0; i < pl->n_pos; ++i) {
                int64_t hq = (int64_t)floor(hx[i]);
                double fr = hx[i] - floor(hx[i]);
                if (hq >= hb - 1 && hq <= hb + 1 && (fr < 1e-6 || fr > 1.0 - 1e-6))
                    pl->near_thresh += 1;
            }
        }
        free(hx);
        free(r);
    } else {
        for (int64_t i = 0; i < pl->n_pos; ++i) {
            admit[i] = 1;
            if (thr >= 0.0) {
                double h = or_entropy_bits(img, N, (int)(i % per) * L, (int)(i / per) * L, 2 * B);
                if (fabs(h - thr) < 1e-9) pl->near_thresh += 1;
                admit[i] = h > thr;
            }
        }
    }
    /* admitted positions in raster order (y first, then x) */
    for (int64_t i = 0; i < pl->n_pos; ++i)
        if (admit[i]) {
            pl->x[pl->dn] = (int32_t)(i % per) * L;
            pl->y[pl->dn] = (int32_t)(i / per) * L;
            pl->dn += 1;
        }
    free(admit);
    size_t cnt = (size_t)(pl->dn ? pl->dn : 1);
    pl->dsum = (int32_t*)malloc(sizeof(int32_t) * cnt * (size_t)n);
    pl->sum_d = (int64_t*)malloc(sizeof(int64_t) * cnt);
    pl->sum_d2 = (int64_t*)malloc(sizeof(int64_t) * cnt);
    if (!pl->dsum || !pl->sum_d || !pl->sum_d2) return -1;
    for (int64_t c = 0; c < pl->dn; ++c) {
        int32_t* d = pl->dsum + (size_t)c * n;
        or_decimate(img, N, pl->x[c], pl->y[c], B, d);
        int64_t s = 0, s2 = 0;
        for (int i = 0; i < n; ++i) { s += d[i]; s2 += (int64_t)d[i] * d[i]; }
        pl->sum_d[c] = s;
        pl->sum_d2[c] = s2;
    }
    return 0;
}

int or_pool_build(const uint8_t* img, int N, int B, int L, double thr, or_pool* pl)
{
    return or_pool_build_ex(img, N, B, L, thr, 0, pl);
}

/* ------------------------------------------------------------------ */
/* Sec. 2 search: best (pool index, isometry, S) for one range.        */
/* Every pool domain, in each of the 8 isometries, at every S of the   */
/* step; lexicographic minimum of (score, pool index, isometry, S).    */
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t score;
    int64_t pool_idx;     /* -1 when the pool is empty */
    int32_t iso, s_idx;
} or_best;

static void read_block(const uint8_t* img, int N, int x, int y, int B, int32_t* r)
{
    for (int i = 0; i < B; ++i)
        for (int j = 0; j < B; ++j)
            r[i * B + j] = img[(y + i) * N + x + j];
}

static or_best search_range(const uint8_t* img, int N, int rx, int ry,
                            const or_pool* pl, const or_sset* ss)
{
    int B = pl->B, n = B * B;
    int32_t r[32 * 32], t[32 * 32];
    read_block(img, N, rx, ry, B, r);
    int64_t sr = 0, sr2 = 0;
    for (int i = 0; i < n; ++i) { sr += r[i]; sr2 += (int64_t)r[i] * r[i]; }
    or_best best = { INT64_MAX, -1, 0, 0 };
    for (int64_t c = 0; c < pl->dn; ++c) {
        const int32_t* d = pl->dsum + (size_t)c * n;
        for (int k = 0; k < 8; ++k) {
            or_isometry(d, B, k, t);
            int64_t srd = 0;
            for (int i = 0; i < n; ++i) srd += (int64_t)r[i] * t[i];
            for (int s = 0; s < ss->n_s; ++s) {
                int64_t sc = score_from_sums(n, sr, sr2, pl->sum_d[c], pl->sum_d2[c],
                                             srd, ss->p[s], ss->q);
                /* strict "<": candidates arrive in increasing (c, k, s). */
                if (sc < best.score) {
                    best.score = sc; best.pool_idx = c; best.iso = k; best.s_idx = s;
                }
            }
        }
    }
    return best;
}

/* Exported single-range search (used for sampled checks and timing). */
int or_search_range(const uint8_t* img, int N, int rx, int ry, const or_pool* pl,
                    const or_sset* ss, int64_t* score, int64_t* pool_idx,
                    int32_t* iso, int32_t* s_idx)
{
    or_best b = search_range(img, N, rx, ry, pl, ss);
    *score = b.score; *pool_idx = b.pool_idx; *iso = b.iso; *s_idx = b.s_idx;
    return 0;
}

/* Many ranges at once, parallel over ranges (results are per range, so the
 * thread count changes nothing but speed). */
int or_search_ranges(const uint8_t* img, int N, int64_t count, const int32_t* rxs,
                     const int32_t* rys, const or_pool* pl, const or_sset* ss,
                     int nthreads, int64_t* score, int64_t* pool_idx, int32_t* iso,
                     int32_t* s_idx)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t i = 0; i < count; ++i) {
        or_best b = search_range(img, N, rxs[i], rys[i], pl, ss);
        score[i] = b.score; pool_idx[i] = b.pool_idx; iso[i] = b.iso; s_idx[i] = b.s_idx;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Sec. 2 quadtree: encode one block, recursing into TL, TR, BL, BR.   */
/* ------------------------------------------------------------------ */
typedef struct {
    or_code* v;
    int64_t n, cap;
} code_list;

static int push_code(code_list* cl, const or_code* c)
{
    if (cl->n == cl->cap) {
        int64_t nc = cl->cap ? 2 * cl->cap : 64;
        or_code* nv = (or_code*)realloc(cl->v, sizeof(or_code) * (size_t)nc);
        if (!nv) return -1;
        cl->v = nv; cl->cap = nc;
    }
    cl->v[cl->n++] = *c;
    return 0;
}

typedef struct {
    const uint8_t* img;
    int N, n_levels, e16;
    const or_pool* pools;     /* one per level */
    const or_sset* ss;        /* one per level */
    int64_t* ranges_searched; /* per level, atomically updated */
} enc_ctx;

static int encode_block(const enc_ctx* e, int x, int y, int level, code_list* out)
{
    const or_pool* pl = &e->pools[level];
    const or_sset* ss = &e->ss[level];
    int B = pl->B;
    int64_t n = (int64_t)B * B;
    int last = (level == e->n_levels - 1);
    int64_t sr = 0;
    for (int i = 0; i < B; ++i)
        for (int j = 0; j < B; ++j) sr += e->img[(y + i) * e->N + x + j];
    int64_t oq = sr / (2 * n);
    if (oq > 127) oq = 127;

    int split = 0;
    if (pl->dn == 0) {
        if (!last) {
            split = 1;
        } else {
            or_code c = { x, y, level, B, 0, -1, (int32_t)oq, 0, 0, 0xFFFFFFFFu, 0 };
            return push_code(out, &c);
        }
    } else {
#ifdef _OPENMP
#pragma omp atomic
#endif
        e->ranges_searched[level] += 1;
        or_best b = search_range(e->img, e->N, x, y, pl, ss);
        /* RMS error sqrt(E/n) > tol  <=>  256 * score > 16 q^2 n^2 e16^2 */
        int64_t q = ss->q;
        split = !last && (256 * b.score > 16 * q * q * n * n * (int64_t)e->e16 * e->e16);
        if (!split) {
            or_code c = { x, y, level, B, b.iso, b.s_idx, (int32_t)oq,
                          pl->x[b.pool_idx], pl->y[b.pool_idx], (uint32_t)b.pool_idx,
                          b.score };
            return push_code(out, &c);
        }
    }
    int h = B / 2;
    if (encode_block(e, x, y, level + 1, out)) return -1;         /* TL */
    if (encode_block(e, x + h, y, level + 1, out)) return -1;     /* TR */
    if (encode_block(e, x, y + h, level + 1, out)) return -1;     /* BL */
    return encode_block(e, x + h, y + h, level + 1, out);         /* BR */
}

/* Per-level counters reported beside the codes. */
typedef struct {
    int32_t n_levels;
    int64_t pool_size[OR_MAX_LEVELS];
    int64_t ranges[OR_MAX_LEVELS];      /* ranges searched at the level */
    int64_t near_thresh[OR_MAX_LEVELS];
} or_stats;

/* Full encoder.  Returns 0, or -1 on bad arguments / allocation failure,
 * or -2 when cap is too small (n_out then holds the needed count). */
int or_encode(const uint8_t* img, int N, int B_max, int B_min, int L, double thr,
              int64_t pool_dn, const or_sset* ss, double tol, int nthreads, or_code* out,
              int64_t cap, int64_t* n_out, or_stats* st)
{
    if (N <= 0 || B_max < B_min || B_min < 1 || L < 1 || B_max > 32) return -1;
    if (N % B_max) return -1;
    int n_levels = 0;
    for (int b = B_max; b >= B_min; b /= 2) {
        if (b % 2 && b != B_min) return -1;
        ++n_levels;
        if (b == B_min) break;
    }
    if ((B_max >> (n_levels - 1)) != B_min || n_levels > OR_MAX_LEVELS) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    or_pool pools[OR_MAX_LEVELS];
    memset(pools, 0, sizeof(pools));
    for (int l = 0; l < n_levels; ++l)
        if (or_pool_build_ex(img, N, B_max >> l, L, thr, pool_dn, &pools[l])) return -1;

    int64_t searched[OR_MAX_LEVELS] = { 0 };
    enc_ctx e = { img, N, n_levels, (int)lround(16.0 * tol), pools, ss, searched };
    int tops = N / B_max;
    int64_t n_top = (int64_t)tops * tops;
    code_list* lists = (code_list*)calloc((size_t)n_top, sizeof(code_list));
    int fail = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t t = 0; t < n_top; ++t) {
        int x = (int)(t % tops) * B_max, y = (int)(t / tops) * B_max;
        if (encode_block(&e, x, y, 0, &lists[t])) fail = 1;
    }
    int64_t total = 0;
    for (int64_t t = 0; t < n_top; ++t) total += lists[t].n;
    *n_out = total;
    int rc = fail ? -1 : (total > cap ? -2 : 0);
    if (rc == 0) {
        int64_t k = 0;
        for (int64_t t = 0; t < n_top; ++t) {
            memcpy(out + k, lists[t].v, sizeof(or_code) * (size_t)lists[t].n);
            k += lists[t].n;
        }
    }
    for (int64_t t = 0; t < n_top; ++t) free(lists[t].v);
    free(lists);
    if (st) {
        memset(st, 0, sizeof(*st));
        st->n_levels = n_levels;
        for (int l = 0; l < n_levels; ++l) {
            st->pool_size[l] = pools[l].dn;
            st->ranges[l] = searched[l];
            st->near_thresh[l] = pools[l].near_thresh;
        }
    }
    for (int l = 0; l < n_levels; ++l) or_pool_free(&pools[l]);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Decoder (Sec. 2: each range rebuilt from its domain and mapping).   */
/* Integer form of r^ = (2 o_q + 1) + S (d - mean(d)), d = T(d')/4,    */
/* rounded half up and clamped to [0, 255].                            */
/* ------------------------------------------------------------------ */
static void apply_code(const or_code* c, const or_sset* ss, const uint8_t* src,
                       int N, uint8_t* dst)
{
    int B = c->B;
    int64_t n = (int64_t)B * B;
    if (c->s_idx < 0) {
        for (int i = 0; i < B; ++i)
            for (int j = 0; j < B; ++j)
                dst[(c->ry + i) * N + c->rx + j] = (uint8_t)(2 * c->o_q + 1);
        return;
    }
    int32_t d[32 * 32], t[32 * 32];
    or_decimate(src, N, c->dx, c->dy, B, d);
    or_isometry(d, B, c->iso, t);
    int64_t sd = 0;
    for (int i = 0; i < n; ++i) sd += d[i];
    int64_t p = ss[c->level].p[c->s_idx], q = ss[c->level].q;
    int64_t den = 4 * q * n;
    for (int i = 0; i < B; ++i)
        for (int j = 0; j < B; ++j) {
            int64_t num = (2 * (int64_t)c->o_q + 1) * den + p * (n * t[i * B + j] - sd) + den / 2;
            int64_t v = num >= 0 ? num / den : -((-num + den - 1) / den);  /* floor */
            if (v < 0) v = 0;
            if (v > 255) v = 255;
            dst[(c->ry + i) * N + c->rx + j] = (uint8_t)v;
        }
}

int or_decode(const or_code* codes, int64_t n_codes, const or_sset* ss, int N,
              int iters_max, uint8_t* out, int* iters_used)
{
    size_t npx = (size_t)N * N;
    uint8_t* cur = (uint8_t*)malloc(npx);
    uint8_t* nxt = (uint8_t*)malloc(npx);
    if (!cur || !nxt) { free(cur); free(nxt); return -1; }
    memset(cur, 128, npx);
    int it = 0;
    for (; it < iters_max; ++it) {
        memcpy(nxt, cur, npx);
        for (int64_t i = 0; i < n_codes; ++i) apply_code(&codes[i], ss, cur, N, nxt);
        int same = memcmp(nxt, cur, npx) == 0;
        uint8_t* tmp = cur; cur = nxt; nxt = tmp;
        if (same) { ++it; break; }
    }
    memcpy(out, cur, npx);
    *iters_used = it;
    free(cur); free(nxt);
    return 0;
}

/* Eq. 4: PSNR in dB between two N x N images (infinity when identical). */
double or_psnr(const uint8_t* a, const uint8_t* b, int64_t npx)
{
    double se = 0.0;
    for (int64_t i = 0; i < npx; ++i) {
        double d = (double)a[i] - (double)b[i];
        se += d * d;
    }
    if (se == 0.0) return INFINITY;
    return 10.0 * log10(255.0 * 255.0 / (se / (double)npx));
}

/* Eq. 8: address width X = ceil(log2 DN) bits. */
int or_address_bits(int64_t dn)
{
    int x = 0;
    while (((int64_t)1 << x) < dn) ++x;
    return x;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Sec. 3.3, Fig. 7, eq. 8: the stored bit stream.                    */
/*                                                                    */
/* Records are stored in their order (top ranges left->right, top->    */
/* bottom, then TL, TR, BL, BR), so range positions are implicit.     */
/* Each record: step (2 bits), range mean (7 bits, o_q), and when the */
/* step's pool is not empty: isometry (3 bits), domain address        */
/* (X = ceil(log2 DN) bits, eq. 8) and the S index (ceil(log2 |S|)    */
/* bits: none for a one-valued set, 1 bit for two values).            */
/* A decoder also needs each step's domain list (the address indexes  */
/* it) and the S sets; they go in a byte-aligned header:              */
/*   "FIC1", u16 N, u8 B_max, u8 steps, u16 L, u8 pool rule (0        */
/*   threshold, 1 top-DN), u32 records; per step: u8 |S|, u16 q,      */
/*   |S| x u16 p, u32 DN (0 when no range reached the step), u8 list  */
/*   form (0: none needed - empty pool or every position; 1: DN       */
/*   positions (x/L, y/L) of ceil(log2 per) bits each; 2: a bitmap of */
/*   the per^2 positions, whichever is shorter, 1 on ties), then the  */
/*   list padded to a byte.  Integers are big-endian; bit fields are  */
/*   written most significant bit first; the payload is padded to a   */
/*   byte at the end.                                                 */
/* ------------------------------------------------------------------ */
typedef struct { uint8_t* buf; int64_t cap, bit; } or_bitw;

static void bw_put(or_bitw* w, uint64_t v, int nb)
{
    for (int i = nb - 1; i >= 0; --i) {
        if (w->buf && (w->bit >> 3) < w->cap) {
            uint8_t* b = &w->buf[w->bit >> 3];
            if ((v >> i) & 1u) *b |= (uint8_t)(0x80u >> (w->bit & 7));
            else *b &= (uint8_t)~(0x80u >> (w->bit & 7));
        }
        w->bit += 1;
    }
}

static void bw_align(or_bitw* w)
{
    while (w->bit & 7) bw_put(w, 0, 1);
}

/* Bytes of the stream (written to out when cap is large enough; the return
 * value is the full size either way), or -1 on bad arguments.  *payload_bits
 * (may be NULL) receives the bits of the records alone.  The pools are
 * rebuilt from img with the encoder's rule. */
int64_t or_pack(const uint8_t* img, int N, int B_max, int n_levels, int L, double thr,
                int64_t pool_dn, const or_sset* ss, const int64_t* searched,
                const or_code* codes, int64_t n, uint8_t* out, int64_t cap,
                int64_t* payload_bits)
{
    if (N <= 0 || N > 65535 || n_levels < 1 || n_levels > 4 || L < 1 || L > 65535) return -1;
    or_bitw w = { out, out ? cap : 0, 0 };
    bw_put(&w, 'F', 8); bw_put(&w, 'I', 8); bw_put(&w, 'C', 8); bw_put(&w, '1', 8);
    bw_put(&w, (uint64_t)N, 16);
    bw_put(&w, (uint64_t)B_max, 8);
    bw_put(&w, (uint64_t)n_levels, 8);
    bw_put(&w, (uint64_t)L, 16);
    bw_put(&w, pool_dn > 0 ? 1u : 0u, 8);
    bw_put(&w, (uint64_t)n, 32);
    int64_t dn[4] = { 0, 0, 0, 0 };
    for (int l = 0; l < n_levels; ++l) {
        const int B = B_max >> l;
        bw_put(&w, (uint64_t)ss[l].n_s, 8);
        bw_put(&w, (uint64_t)ss[l].q, 16);
        for (int i = 0; i < ss[l].n_s; ++i) bw_put(&w, (uint64_t)ss[l].p[i], 16);
        or_pool pl;
        memset(&pl, 0, sizeof(pl));
        if (searched[l] > 0) {
            if (or_pool_build_ex(img, N, B, L, thr, pool_dn, &pl)) return -1;
            dn[l] = pl.dn;
        }
        const int per = or_positions_per_axis(N, B, L);
        const int64_t npos = (int64_t)per * per;
        bw_put(&w, (uint64_t)dn[l], 32);
        int form = 0;
        const int pw = or_address_bits(per);
        if (dn[l] > 0 && dn[l] < npos) form = (dn[l] * 2 * pw <= npos) ? 1 : 2;
        bw_put(&w, (uint64_t)form, 8);
        if (form == 1) {
            for (int64_t c = 0; c < dn[l]; ++c) {
                bw_put(&w, (uint64_t)(pl.x[c] / L), pw);
                bw_put(&w, (uint64_t)(pl.y[c] / L), pw);
            }
        } else if (form == 2) {
            int64_t c = 0;
            for (int64_t i = 0; i < npos; ++i) {
                const int x = (int)(i % per) * L, y = (int)(i / per) * L;
                const int in = c < dn[l] && pl.x[c] == x && pl.y[c] == y;
                if (in) ++c;
                bw_put(&w, in ? 1u : 0u, 1);
            }
        }
        bw_align(&w);
        if (searched[l] > 0) or_pool_free(&pl);
    }
    const int64_t head = w.bit;
    for (int64_t i = 0; i < n; ++i) {
        const or_code* c = &codes[i];
        const int l = c->level;
        if (l < 0 || l >= n_levels) return -1;
        bw_put(&w, (uint64_t)l, 2);
        bw_put(&w, (uint64_t)c->o_q, 7);
        if (dn[l] > 0) {
            bw_put(&w, (uint64_t)c->iso, 3);
            bw_put(&w, (uint64_t)c->pool_idx, or_address_bits(dn[l]));
            bw_put(&w, (uint64_t)c->s_idx, or_address_bits(ss[l].n_s));
        }
    }
    if (payload_bits) *payload_bits = w.bit - head;
    bw_align(&w);
    return w.bit >> 3;
}

typedef struct { const uint8_t* buf; int64_t n, bit; int bad; } or_bitr;

static uint64_t br_get(or_bitr* r, int nb)
{
    uint64_t v = 0;
    for (int i = 0; i < nb; ++i) {
        if ((r->bit >> 3) >= r->n) { r->bad = 1; return 0; }
        v = (v << 1) | ((r->buf[r->bit >> 3] >> (7 - (r->bit & 7))) & 1u);
        r->bit += 1;
    }
    return v;
}

typedef struct {
    or_bitr* r;
    int B_max, n_levels, L, N;
    int64_t dn[4];
    int per[4];
    int32_t* lx[4];
    int32_t* ly[4];
    const or_sset* ss;
    or_code* out;
    int64_t cap, n;
    uint64_t pending;  /* step of the record read ahead, or ~0 */
} or_unpack_ctx;

static int unpack_block(or_unpack_ctx* u, int x, int y, int lvl)
{
    if (lvl >= u->n_levels) return -1;
    if (u->pending == ~(uint64_t)0) u->pending = br_get(u->r, 2);
    if (u->r->bad) return -1;
    if ((int)u->pending > lvl) {
        const int h = (u->B_max >> lvl) / 2;
        if (unpack_block(u, x, y, lvl + 1) || unpack_block(u, x + h, y, lvl + 1) ||
            unpack_block(u, x, y + h, lvl + 1) || unpack_block(u, x + h, y + h, lvl + 1))
            return -1;
        return 0;
    }
    if ((int)u->pending != lvl) return -1;
    u->pending = ~(uint64_t)0;
    or_code c;
    memset(&c, 0, sizeof(c));
    c.rx = x; c.ry = y; c.level = lvl; c.B = u->B_max >> lvl;
    c.o_q = (int32_t)br_get(u->r, 7);
    if (u->dn[lvl] > 0) {
        c.iso = (int32_t)br_get(u->r, 3);
        c.pool_idx = (uint32_t)br_get(u->r, or_address_bits(u->dn[lvl]));
        c.s_idx = (int32_t)br_get(u->r, or_address_bits(u->ss[lvl].n_s));
        if ((int64_t)c.pool_idx >= u->dn[lvl]) return -1;
        c.dx = u->lx[lvl][c.pool_idx];
        c.dy = u->ly[lvl][c.pool_idx];
    } else {
        c.s_idx = -1;
        c.pool_idx = 0xFFFFFFFFu;
    }
    if (u->r->bad) return -1;
    if (u->n < u->cap) u->out[u->n] = c;
    u->n += 1;
    return 0;
}

/* Reads a stream written by or_pack.  Returns 0, -1 on a malformed stream,
 * -2 when cap is too small (*n_out then holds the count).  ss_out receives
 * the S sets (4 entries), *N_out, *B_max_out, *n_levels_out the geometry. */
int or_unpack(const uint8_t* in, int64_t nbytes, or_code* out, int64_t cap, int64_t* n_out,
              or_sset* ss_out, int* N_out, int* B_max_out, int* n_levels_out)
{
    or_bitr r = { in, nbytes, 0, 0 };
    if (br_get(&r, 32) != (((uint64_t)'F' << 24) | ((uint64_t)'I' << 16) | ((uint64_t)'C' << 8) | '1'))
        return -1;
    or_unpack_ctx u;
    memset(&u, 0, sizeof(u));
    u.r = &r;
    u.N = (int)br_get(&r, 16);
    u.B_max = (int)br_get(&r, 8);
    u.n_levels = (int)br_get(&r, 8);
    u.L = (int)br_get(&r, 16);
    (void)br_get(&r, 8);
    const int64_t n_codes = (int64_t)br_get(&r, 32);
    if (r.bad || u.n_levels < 1 || u.n_levels > 4 || u.L < 1 || u.B_max < 1 || u.N % u.B_max)
        return -1;
    memset(ss_out, 0, sizeof(or_sset) * 4);
    int rc = 0;
    for (int l = 0; l < u.n_levels && !rc; ++l) {
        const int B = u.B_max >> l;
        ss_out[l].n_s = (int)br_get(&r, 8);
        ss_out[l].q = (int)br_get(&r, 16);
        if (ss_out[l].n_s > OR_MAX_S) { rc = -1; break; }
        for (int i = 0; i < ss_out[l].n_s; ++i) ss_out[l].p[i] = (int)br_get(&r, 16);
        u.dn[l] = (int64_t)br_get(&r, 32);
        const int form = (int)br_get(&r, 8);
        const int per = or_positions_per_axis(u.N, B, u.L);
        const int64_t npos = (int64_t)per * per;
        const int pw = or_address_bits(per);
        u.per[l] = per;
        if (u.dn[l] > npos) { rc = -1; break; }
        u.lx[l] = (int32_t*)malloc(sizeof(int32_t) * (size_t)(u.dn[l] ? u.dn[l] : 1));
        u.ly[l] = (int32_t*)malloc(sizeof(int32_t) * (size_t)(u.dn[l] ? u.dn[l] : 1));
        if (!u.lx[l] || !u.ly[l]) { rc = -1; break; }
        if (form == 0) {
            if (u.dn[l] != 0 && u.dn[l] != npos) { rc = -1; break; }
            for (int64_t i = 0; i < u.dn[l]; ++i) {
                u.lx[l][i] = (int32_t)(i % per) * u.L;
                u.ly[l][i] = (int32_t)(i / per) * u.L;
            }
        } else if (form == 1) {
            for (int64_t i = 0; i < u.dn[l]; ++i) {
                u.lx[l][i] = (int32_t)br_get(&r, pw) * u.L;
                u.ly[l][i] = (int32_t)br_get(&r, pw) * u.L;
            }
        } else if (form == 2) {
            int64_t c = 0;
            for (int64_t i = 0; i < npos; ++i)
                if (br_get(&r, 1)) {
                    if (c >= u.dn[l]) { rc = -1; break; }
                    u.lx[l][c] = (int32_t)(i % per) * u.L;
                    u.ly[l][c] = (int32_t)(i / per) * u.L;
                    ++c;
                }
            if (!rc && c != u.dn[l]) rc = -1;
        } else {
            rc = -1;
        }
        while (r.bit & 7) (void)br_get(&r, 1);
    }
    if (!rc) {
        u.ss = ss_out;
        u.out = out;
        u.cap = cap;
        u.pending = ~(uint64_t)0;
        const int tops = u.N / u.B_max;
        for (int t = 0; t < tops * tops && !rc; ++t)
            rc = unpack_block(&u, (t % tops) * u.B_max, (t / tops) * u.B_max, 0);
        if (!rc && (r.bad || u.n != n_codes)) rc = -1;
    }
    for (int l = 0; l < 4; ++l) { free(u.lx[l]); free(u.ly[l]); }
    *n_out = u.n;
    *N_out = u.N;
    *B_max_out = u.B_max;
    *n_levels_out = u.n_levels;
    if (rc) return rc;
    return u.n > cap ? -2 : 0;
}
