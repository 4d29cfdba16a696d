/*
 * CPU oracle for dynamic tile / rectangular-slice (TRS) frame partitioning,
 * "Quality-driven Dynamic VVC Frame Partitioning for efficient Parallel
 * Processing" (Amestoy, Hamidouche, Bergeron, Menard, ICIP 2020).
 *
 * TEST INFRASTRUCTURE.  This file is the plain, slow reference that the CUDA
 * library is checked against.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the library never does.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * Contents, each following the passage cited beside it:
 *   oracle_texture      per-CTU luma sums S1 = sum p, S2 = sum p^2, N     (Sec. 2.2, Eq. 2),
 *                       from 8..12-bit samples or the packed 10-bit format
 *   oracle_time_q       Q16 fixed-point CTU times                          (Sec. 2.1, Eq. 1 input)
 *   oracle_sat          summed-area table by its definition (direct sums)
 *   oracle_search_enum  O1: every TRS configuration enumerated in canonical
 *                       code order, evaluated by direct sums (a partial
 *                       configuration is not extended once it breaks the area
 *                       rule or Eq. 4, or leaves a rest of the frame the other
 *                       slices cannot fill under the rule: no completion of it
 *                       is valid):
 *                       step 1 T_min (Eq. 3), step 2 arg-min of Eq. 2 under
 *                       Eq. 4, both under k*A_min > A_max (Sec. 2.3)
 *   oracle_search_dp    O2: exact dynamic programme over the same space;
 *                       equal to O1 by construction (checked by the tests)
 *   oracle_search_dp_windows  O2 over every s-th area window only (the
 *                       lighter search the paper leaves to future work, Sec. 4)
 *   oracle_mt_search    the multi-tile slice space (slices of one tile or
 *                       rectangles of whole tiles), enumerated (Sec. 1, Fig. 1b):
 *                       every tile grid, its tiles grouped into rectangles
 *   oracle_mt_count     the number of distinct slice sets of that space
 *   oracle_mt_search_rects  the same search over the partitions of the CTU
 *                       grid into n rectangles (the same space), reaching
 *                       full frame sizes for small n
 *   oracle_evaluate,    T, Q and the area extremes of a given partition or
 *   oracle_rect,        rectangle, or of every CTU rectangle, by direct sums
 *   oracle_rect_all     (checkers for the tests)
 *
 * Every function is pinned by the tests against what the paper and the
 * mathematics fix, not against itself: brute force over all line subsets or
 * all rectangle partitions on tiny frames, closed-form counts, constant and
 * ramp planes, hand-worked cases, exact rational SSE from the samples.
 * tests/test_oracle_mutants.py plants slips in a copy of this file and
 * checks that each one fails a pin.
 *
 * Readings of the paper used here (the paper is silent on these points):
 *   - CTUs are 128x128 luma samples; edge CTUs are clipped to the frame.
 *   - A partition has exactly n rectangular slices (one per thread, Sec. 2.1).
 *     A slice is a run of complete CTU rows inside one tile (Sec. 1); tiles
 *     form a grid on CTU lines; every tile holds >= 1 slice.
 *   - "Area" in k*A_min > A_max counts luma samples; k = 3; strict '>'.
 *     The rule applies to both search steps.
 *   - Times are quantised to Q16: Tq = rint(t * 65536), t finite, 0 <= t < 65536.
 *   - lambda_q = rint(lambda * 65536); Eq. 4 is tested as
 *     T(P) * 65536 <= T_min * (65536 + lambda_q), inclusive.
 *   - The quality term of a slice is the floor of its exact luma SSE,
 *     S2 - ceil(S1^2 / N); Q(P) is the sum over slices.
 *   - Ties on Q are broken by the smallest canonical code: the tile-row cut
 *     bits top to bottom, then per tile column left to right its right edge
 *     followed by the in-tile slice cut bits of its tiles top to bottom
 *     ('0' < '1').  In the multi-tile space, by the smallest list of slices in
 *     raster order of their top-left corners, each compared as
 *     (y0, x0, y1, x1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

#define OR_CTU 128
#define OR_MAX_C 64
#define OR_MAX_R 64
#define OR_MAX_N 64
#define OR_INF UINT64_MAX
#define OR_PACKED10 0x10A  /* the packed 10-bit sample format's code in the library's interface */

enum { OR_OK = 0, OR_EINVAL = 1, OR_ERANGE = 2, OR_EINFEASIBLE = 3, OR_ENOMEM = 4 };

typedef struct {
    int status;
    int n;              /* number of rectangular slices */
    int c;              /* tile columns */
    int r;              /* tile rows */
    uint64_t row_mask;  /* tile-row cuts: bit (y-1) set => tile boundary at CTU line y */
    int x_edges[OR_MAX_C + 1];      /* tile column edges, x_edges[0]=0 .. x_edges[c]=C */
    uint64_t band_cuts[OR_MAX_C];   /* per tile column: every horizontal slice boundary */
    uint64_t t_min;     /* Eq. 3, Q16 */
    uint64_t thr;       /* largest T(P) allowed by Eq. 4 */
    uint64_t t;         /* T(P*) */
    uint64_t q;         /* Q(P*) */
    uint64_t n_candidates;   /* configurations reached (O1; all of S(n) with the area rule off) */
    uint64_t n_valid;        /* of those, passing the area rule (O1) */
    uint64_t n_windows;      /* area windows examined (O2) */
    double t_real, t_min_real, sse_real;
} oracle_result;

/* ------------------------------------------------------------------ */
/* Frame geometry                                                      */

typedef struct {
    int W, H, C, R;
    const uint64_t *S1, *S2, *N;   /* per CTU, row-major R x C */
    const uint32_t *Tq;            /* per CTU, Q16 */
} frame_t;

static int ctu_w(const frame_t *f, int x) {
    int e = (x + 1) * OR_CTU;
    return (e <= f->W ? e : f->W) - x * OR_CTU;
}
static int ctu_h(const frame_t *f, int y) {
    int e = (y + 1) * OR_CTU;
    return (e <= f->H ? e : f->H) - y * OR_CTU;
}

/* Sums over the CTUs of rectangle [x0,x1) x [y0,y1), by direct loops. */
typedef struct { uint64_t T, S1, S2, N; } rsum_t;

static rsum_t rect_direct(const frame_t *f, int x0, int x1, int y0, int y1) {
    rsum_t s = {0, 0, 0, 0};
    for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) {
            int i = y * f->C + x;
            s.T += f->Tq[i];
            s.S1 += f->S1[i];
            s.S2 += f->S2[i];
            s.N += f->N[i];
        }
    return s;
}

/* Floor of the exact SSE of a region: S2 - ceil(S1^2 / N)  (Eq. 2 summand). */
static uint64_t sse_floor(uint64_t S1, uint64_t S2, uint64_t N) {
    u128 sq = (u128)S1 * (u128)S1;
    u128 c = (sq + (u128)(N - 1)) / (u128)N;
    return S2 - (uint64_t)c;
}

static long double sse_exact(uint64_t S1, uint64_t S2, uint64_t N) {
    return (long double)S2 - ((long double)S1 * (long double)S1) / (long double)N;
}

/* Memo of rectangle sums keyed by (x0,x1,y0,y1); each entry filled by rect_direct. */
typedef struct {
    const frame_t *f;
    rsum_t *tab;
    uint8_t *have;
} memo_t;

static size_t memo_idx(const frame_t *f, int x0, int x1, int y0, int y1) {
    return (((size_t)x0 * (f->C + 1) + x1) * (f->R + 1) + y0) * (f->R + 1) + y1;
}

static int memo_init(memo_t *m, const frame_t *f) {
    size_t n = (size_t)(f->C + 1) * (f->C + 1) * (f->R + 1) * (f->R + 1);
    m->f = f;
    m->tab = (rsum_t *)malloc(n * sizeof(rsum_t));
    m->have = (uint8_t *)calloc(n, 1);
    return (m->tab && m->have) ? 0 : -1;
}
static void memo_free(memo_t *m) {
    free(m->tab);
    free(m->have);
}
static rsum_t memo_get(memo_t *m, int x0, int x1, int y0, int y1) {
    size_t i = memo_idx(m->f, x0, x1, y0, y1);
    if (!m->have[i]) {
        m->tab[i] = rect_direct(m->f, x0, x1, y0, y1);
        m->have[i] = 1;
    }
    return m->tab[i];
}

/* ------------------------------------------------------------------ */
/* a1: per-CTU texture statistics (Eq. 2 needs sum p and sum p^2 per RS) */

/* bd: 8..12, or OR_PACKED10 for 10-bit samples packed four in five bytes,
   each row a little-endian bit string with sample x in bits [10x, 10x+10). */
int oracle_texture(const void *luma, int W, int H, size_t pitch, int bd,
                   uint64_t *S1, uint64_t *S2, uint64_t *N, uint32_t *vmax) {
    int packed = bd == OR_PACKED10;
    if (packed) bd = 10;
    if (!luma || W <= 0 || H <= 0 || bd < 8 || bd > 12) return OR_EINVAL;
    int bps = (bd == 8) ? 1 : 2;
    size_t row_bytes = packed ? ((size_t)W * 10 + 7) / 8 : (size_t)W * bps;
    if (pitch < row_bytes) return OR_EINVAL;
    int C = (W + OR_CTU - 1) / OR_CTU, R = (H + OR_CTU - 1) / OR_CTU;
    for (int i = 0; i < C * R; ++i) {
        S1[i] = 0;
        S2[i] = 0;
        N[i] = 0;
        vmax[i] = 0;
    }
    int bad = 0;
    const uint8_t *base = (const uint8_t *)luma;
    for (int y = 0; y < H; ++y) {
        const uint8_t *row = base + (size_t)y * pitch;
        for (int x = 0; x < W; ++x) {
            uint32_t p;
            if (packed) {
                p = 0;
                for (int i = 0; i < 10; ++i) {
                    size_t bit = (size_t)10 * x + i;
                    p |= (uint32_t)((row[bit >> 3] >> (bit & 7)) & 1u) << i;
                }
            } else if (bps == 1) {
                p = row[x];
            } else {
                p = (uint32_t)row[2 * x] | ((uint32_t)row[2 * x + 1] << 8); /* little endian */
            }
            int i = (y / OR_CTU) * C + (x / OR_CTU);
            S1[i] += p;
            S2[i] += (uint64_t)p * p;
            N[i] += 1;
            if (p > vmax[i]) vmax[i] = p;
            if (p >> bd) bad = 1;
        }
    }
    return bad ? OR_ERANGE : OR_OK;
}

/* ------------------------------------------------------------------ */
/* a2 inputs: Q16 CTU times (estimator values of Sec. 2.1)             */

int oracle_time_q(const float *t, int count, uint32_t *Tq) {
    int bad = 0;
    for (int i = 0; i < count; ++i) {
        double v = (double)t[i];
        if (!(v >= 0.0) || !(v < 65536.0)) {
            Tq[i] = 0;
            bad = 1;
            continue;
        }
        Tq[i] = (uint32_t)rint(v * 65536.0);
    }
    return bad ? OR_ERANGE : OR_OK;
}

uint32_t oracle_lambda_q(float lambda) { return (uint32_t)rint((double)lambda * 65536.0); }

/* Summed-area table by definition: sat[y][x] = sum of v over [0,x) x [0,y). */
void oracle_sat(const uint64_t *v, int C, int R, uint64_t *sat) {
    for (int y = 0; y <= R; ++y)
        for (int x = 0; x <= C; ++x) {
            uint64_t s = 0;
            for (int yy = 0; yy < y; ++yy)
                for (int xx = 0; xx < x; ++xx) s += v[yy * C + xx];
            sat[y * (C + 1) + x] = s;
        }
}

/* ------------------------------------------------------------------ */
/* Shared pieces of both searches                                       */

static int check_inputs(int W, int H, int n, int k_area) {
    if (W <= 0 || H <= 0 || n < 1 || n > OR_MAX_N || k_area < 1) return OR_EINVAL;
    int C = (W + OR_CTU - 1) / OR_CTU, R = (H + OR_CTU - 1) / OR_CTU;
    if (C > OR_MAX_C || R > OR_MAX_R) return OR_EINVAL;
    return OR_OK;
}

/* Eq. 4 bound as the largest integer T with T*65536 <= T_min*(65536+lambda_q). */
static uint64_t eq4_thr(uint64_t t_min, uint32_t lambda_q) {
    u128 v = (u128)t_min * (u128)(65536u + (u128)lambda_q);
    u128 q = v / 65536u;
    return q > (u128)UINT64_MAX ? UINT64_MAX : (uint64_t)q;
}

static void fill_reporting(const frame_t *f, memo_t *m, oracle_result *res) {
    long double sse = 0.0L;
    for (int b = 0; b < res->c; ++b) {
        int y0 = 0;
        for (int y = 1; y <= f->R; ++y) {
            if (y == f->R || ((res->band_cuts[b] >> (y - 1)) & 1u)) {
                rsum_t s = memo_get(m, res->x_edges[b], res->x_edges[b + 1], y0, y);
                sse += sse_exact(s.S1, s.S2, s.N);
                y0 = y;
            }
        }
    }
    res->sse_real = (double)sse;
    res->t_real = (double)res->t / 65536.0;
    res->t_min_real = (double)res->t_min / 65536.0;
}

/* ------------------------------------------------------------------ */
/* O1: plain enumeration of every TRS configuration in code order       */

/*
 * A configuration is built band by band (tile columns left to right) and,
 * inside a band, CTU line by CTU line top to bottom: a tile-row line is
 * always a slice boundary, a free line is tried uncut ('0') before cut
 * ('1').  That is the canonical code order, so the first configuration met
 * with the smallest Q is the one with the smallest code.
 *
 * Adding a slice never raises the smallest slice area, never lowers the
 * largest one and never lowers the largest slice time.  So once the slices
 * chosen so far break the area rule (Sec. 2.3), or in step 2 the Eq. 4
 * bound, no completion of them is in S(n) or feasible, and the enumeration
 * does not descend further there.  Nothing that can be valid is skipped and
 * the order of the rest is unchanged.  With the area rule off nothing is
 * skipped in step 1, so the configurations reached are all of S(n).
 */
typedef struct {
    uint64_t amin, amax;  /* smallest and largest slice area so far */
    uint64_t tmax;        /* slowest slice so far (Eq. 1) */
    uint64_t q;           /* sum of the slices' floored SSE so far (Eq. 2) */
} partial_t;

typedef struct {
    const frame_t *f;
    memo_t *memo;
    int n, k_area, area_rule, pass;
    uint64_t row_mask;           /* current tile-row cut lines */
    int r;                       /* tile rows */
    int nb;                      /* bands chosen so far */
    int x_edges[OR_MAX_C + 1];
    uint64_t band_cuts[OR_MAX_C];
    /* results */
    uint64_t t_min, thr;
    uint32_t lambda_q;
    uint64_t best_q;
    int have_best;
    oracle_result *res;
    uint64_t n_candidates, n_valid;
} enum_t;

/* The area rule k*A_min > A_max (Sec. 2.3) on the slices chosen so far. */
static int area_ok(const enum_t *e, const partial_t *p) {
    return !e->area_rule || (u128)e->k_area * p->amin > (u128)p->amax;
}

/* Eq. 4 as printed, T(P) <= T_min * (1 + lambda), in Q16 integers (step 2 only). */
static int eq4_ok(const enum_t *e, const partial_t *p) {
    return e->pass == 1 || (u128)p->tmax * 65536u <= (u128)e->t_min * (65536u + (u128)e->lambda_q);
}

/* p plus the slice [x0,x1) x [y0,y1), its sums taken directly. */
static partial_t add_slice(enum_t *e, partial_t p, int x0, int x1, int y0, int y1) {
    rsum_t s = memo_get(e->memo, x0, x1, y0, y1);
    if (s.N < p.amin) p.amin = s.N;
    if (s.N > p.amax) p.amax = s.N;
    if (s.T > p.tmax) p.tmax = s.T;
    p.q += sse_floor(s.S1, s.S2, s.N);
    return p;
}

/* Whether the n - used slices still to come can fill the columns [x1, C)
   under the area rule: each of them must have an area s with
   k*s > A_max and s < k*A_min of the slices so far, and together they
   cover the rest of the frame exactly. */
static int rest_fits(const enum_t *e, const partial_t *p, int x1, int used) {
    if (!e->area_rule) return 1;
    const frame_t *f = e->f;
    int wpx = (x1 * OR_CTU < f->W ? x1 * OR_CTU : f->W);
    u128 rest = (u128)(uint64_t)(f->W - wpx) * (u128)(uint64_t)f->H;
    u128 left = (u128)(uint64_t)(e->n - used);
    if (left == 0) return rest == 0;
    return (u128)e->k_area * rest > left * p->amax && rest < left * (u128)e->k_area * p->amin;
}

static void enum_evaluate(enum_t *e, const partial_t *p) {
    e->n_candidates++;
    if (!area_ok(e, p)) return;
    e->n_valid++;
    if (e->pass == 1) {
        if (p->tmax < e->t_min) e->t_min = p->tmax;
        return;
    }
    /* pass 2: feasible under Eq. 4, then the first (= lex-smallest code) minimum of Q */
    if (!eq4_ok(e, p)) return;
    if (!e->have_best || p->q < e->best_q) {
        e->have_best = 1;
        e->best_q = p->q;
        oracle_result *r = e->res;
        r->c = e->nb;
        r->r = e->r;
        r->row_mask = e->row_mask;
        for (int b = 0; b <= e->nb; ++b) r->x_edges[b] = e->x_edges[b];
        for (int b = 0; b < e->nb; ++b) r->band_cuts[b] = e->band_cuts[b];
        r->t = p->tmax;
        r->q = p->q;
    }
}

static void enum_bands(enum_t *e, int x, int used, partial_t p);

/* Band [x, x1), CTU line y (1..R-1) and below.  y0 is the top row of the
   open slice, cuts the band's slice boundaries so far and k its slices
   counting the open one and one per tile row below it. */
static void enum_lines(enum_t *e, int x, int x1, int y, int y0, uint64_t cuts, int k, int used, partial_t p) {
    const frame_t *f = e->f;
    if (used + k > e->n) return;  /* more than n slices */
    if (y == f->R) {
        partial_t c = add_slice(e, p, x, x1, y0, f->R);
        if (!area_ok(e, &c) || !eq4_ok(e, &c) || !rest_fits(e, &c, x1, used + k)) return;
        e->x_edges[e->nb + 1] = x1;
        e->band_cuts[e->nb] = cuts;
        e->nb++;
        enum_bands(e, x1, used + k, c);
        e->nb--;
        return;
    }
    int tile_row = (int)((e->row_mask >> (y - 1)) & 1u);
    if (!tile_row) enum_lines(e, x, x1, y + 1, y0, cuts, k, used, p); /* '0': no cut at line y */
    partial_t c = add_slice(e, p, x, x1, y0, y);                      /* '1': slice [y0, y) ends */
    if (!area_ok(e, &c) || !eq4_ok(e, &c)) return;
    enum_lines(e, x, x1, y + 1, y, cuts | (1ull << (y - 1)), tile_row ? k : k + 1, used, c);
}

static void enum_bands(enum_t *e, int x, int used, partial_t p) {
    const frame_t *f = e->f;
    if (x == f->C) {
        if (used == e->n) enum_evaluate(e, &p);
        return;
    }
    if (used + e->r > e->n) return; /* every further tile column holds >= r slices */
    for (int x1 = x + 1; x1 <= f->C; ++x1) enum_lines(e, x, x1, 1, 0, 0, e->r, used, p);
}

static void enum_all(enum_t *e) {
    const frame_t *f = e->f;
    int L = f->R - 1;
    uint64_t lim = 1ull << L;
    for (uint64_t v = 0; v < lim; ++v) {
        /* tile-row cut bits, line 1 most significant */
        e->row_mask = 0;
        e->r = 1;
        for (int y = 1; y <= L; ++y) {
            if ((v >> (L - y)) & 1u) {
                e->row_mask |= 1ull << (y - 1);
                e->r++;
            }
        }
        if (e->r > e->n) continue;
        e->nb = 0;
        e->x_edges[0] = 0;
        partial_t p = {OR_INF, 0, 0, 0};
        enum_bands(e, 0, 0, p);
    }
}

/*
 * O1.  Enumerates S(n) literally: tile rows, tile columns, in-tile slice cuts,
 * exactly n slices, the k*A_min > A_max rule (Sec. 2.3) when area_rule != 0.
 * Step 1 (Eq. 3) and step 2 (Eq. 2 under Eq. 4) are two passes over the same
 * enumeration.  Exponential in n: with the rule on it reaches 1920x1080 with
 * n = 12 (8.6e6 valid configurations) and 3840x2160 with n = 8 (8.9e6), each
 * in seconds; 3840x2160 with n = 16 (3.6e12) is out of its reach.
 */
int oracle_search_enum(int W, int H, const uint64_t *S1, const uint64_t *S2, const uint64_t *N,
                       const uint32_t *Tq, int n, int k_area, uint32_t lambda_q, int area_rule,
                       oracle_result *res) {
    memset(res, 0, sizeof(*res));
    int st = check_inputs(W, H, n, k_area);
    if (st) {
        res->status = st;
        return st;
    }
    frame_t f = {W, H, (W + OR_CTU - 1) / OR_CTU, (H + OR_CTU - 1) / OR_CTU, S1, S2, N, Tq};
    memo_t m;
    if (memo_init(&m, &f)) {
        memo_free(&m);
        res->status = OR_ENOMEM;
        return OR_ENOMEM;
    }
    enum_t e;
    memset(&e, 0, sizeof(e));
    e.f = &f;
    e.memo = &m;
    e.n = n;
    e.k_area = k_area;
    e.area_rule = area_rule;
    e.res = res;
    e.t_min = OR_INF;
    e.pass = 1;
    enum_all(&e);
    res->n_candidates = e.n_candidates;
    res->n_valid = e.n_valid;
    res->n = n;
    if (e.t_min == OR_INF) {
        res->status = OR_EINFEASIBLE;
        memo_free(&m);
        return OR_EINFEASIBLE;
    }
    e.thr = eq4_thr(e.t_min, lambda_q);
    e.lambda_q = lambda_q;
    e.pass = 2;
    e.n_candidates = 0;
    e.n_valid = 0;
    enum_all(&e);
    res->t_min = e.t_min;
    res->thr = e.thr;
    fill_reporting(&f, &m, res);
    memo_free(&m);
    res->status = OR_OK;
    return OR_OK;
}

/* Counts the configurations of S(n) (no objective); a test of the enumerator. */
int oracle_count_enum(int W, int H, int n, int k_area, int area_rule, uint64_t *count) {
    int st = check_inputs(W, H, n, k_area);
    if (st) return st;
    int C = (W + OR_CTU - 1) / OR_CTU, R = (H + OR_CTU - 1) / OR_CTU;
    size_t cells = (size_t)C * R;
    uint64_t *S = (uint64_t *)calloc(cells, sizeof(uint64_t));
    uint64_t *Nn = (uint64_t *)calloc(cells, sizeof(uint64_t));
    uint32_t *T = (uint32_t *)calloc(cells, sizeof(uint32_t));
    if (!S || !Nn || !T) {
        free(S);
        free(Nn);
        free(T);
        return OR_ENOMEM;
    }
    frame_t f = {W, H, C, R, S, S, Nn, T};
    for (int y = 0; y < R; ++y)
        for (int x = 0; x < C; ++x) Nn[y * C + x] = (uint64_t)ctu_w(&f, x) * ctu_h(&f, y);
    memo_t m;
    if (memo_init(&m, &f)) {
        memo_free(&m);
        free(S);
        free(Nn);
        free(T);
        return OR_ENOMEM;
    }
    oracle_result res;
    enum_t e;
    memset(&e, 0, sizeof(e));
    e.f = &f;
    e.memo = &m;
    e.n = n;
    e.k_area = k_area;
    e.area_rule = area_rule;
    e.res = &res;
    e.t_min = OR_INF;
    e.pass = 1;
    enum_all(&e);
    *count = area_rule ? e.n_valid : e.n_candidates;
    memo_free(&m);
    free(S);
    free(Nn);
    free(T);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* O2: exact dynamic programme                                          */
/*
 * Two facts make the search decomposable.
 *
 * (i) Tile rows add no geometry.  A tile-row cut at line y forces a slice
 *     boundary at y in every tile column; the same slices are reached with no
 *     tile-row cut by cutting at y inside each tile.  So every partition of
 *     S(n) is also a partition with a single tile row, and since that
 *     configuration's code starts with all-zero tile-row bits it is the
 *     smallest code of its geometry.  The search therefore runs over tile
 *     columns, each split into horizontal slices.
 *
 * (ii) The area rule becomes local through windows.  If 3*A_min > A_max then
 *     every slice area lies in [a, 3a-1] with a = A_min; conversely if every
 *     area lies in [a, 3a-1] the rule holds.  So S(n) is the union over the
 *     distinct slice areas a of the partitions whose slices all lie in the
 *     window [a, k*a-1].  Within a window, max (Eq. 1) and sum (Eq. 2) are
 *     separable over tile columns and, inside a column, over slices.
 *
 * Per window: step 1 is a min-max DP, step 2 a min-sum DP over slices that
 * also satisfy T(s) <= thr (max over slices <= thr iff each slice <= thr).
 * The lex-smallest code among the minimisers is rebuilt from suffix tables.
 */

typedef struct {
    const frame_t *f;
    memo_t *memo;
    int n, k_area;
    uint64_t a_lo, a_hi;  /* window */
    uint64_t thr;         /* step 2 only */
} dpctx_t;

static int strip_ok(const dpctx_t *d, rsum_t s, int step) {
    if (s.N < d->a_lo || s.N > d->a_hi) return 0;
    if (step == 2 && s.T > d->thr) return 0;
    return 1;
}

/* Step 1, one band [x0,x1): V[k] = min over k-slice splits of the max slice time. */
static void band_minmax(const dpctx_t *d, int x0, int x1, uint64_t *V /* [n+1] */) {
    const frame_t *f = d->f;
    int R = f->R, n = d->n;
    /* G[y][k]: rows [0,y) split into k slices */
    uint64_t G[OR_MAX_R + 1][OR_MAX_N + 1];
    for (int y = 0; y <= R; ++y)
        for (int k = 0; k <= n; ++k) G[y][k] = OR_INF;
    G[0][0] = 0;
    for (int y = 1; y <= R; ++y)
        for (int yp = 0; yp < y; ++yp) {
            rsum_t s = memo_get(d->memo, x0, x1, yp, y);
            if (!strip_ok(d, s, 1)) continue;
            for (int k = 1; k <= n; ++k) {
                if (G[yp][k - 1] == OR_INF) continue;
                uint64_t v = G[yp][k - 1] > s.T ? G[yp][k - 1] : s.T;
                if (v < G[y][k]) G[y][k] = v;
            }
        }
    for (int k = 0; k <= n; ++k) V[k] = G[R][k];
}

static uint64_t window_tmin(const dpctx_t *d) {
    const frame_t *f = d->f;
    int C = f->C, n = d->n;
    uint64_t *V = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(C + 1) * (C + 1) * (n + 1));
    if (!V) return OR_INF;
    for (int x0 = 0; x0 < C; ++x0)
        for (int x1 = x0 + 1; x1 <= C; ++x1)
            band_minmax(d, x0, x1, V + ((size_t)x0 * (C + 1) + x1) * (n + 1));
    /* F[x][m]: columns [0,x) with m slices */
    uint64_t F[OR_MAX_C + 1][OR_MAX_N + 1];
    for (int x = 0; x <= C; ++x)
        for (int m = 0; m <= n; ++m) F[x][m] = OR_INF;
    F[0][0] = 0;
    for (int x = 1; x <= C; ++x)
        for (int xp = 0; xp < x; ++xp) {
            const uint64_t *Vb = V + ((size_t)xp * (C + 1) + x) * (n + 1);
            for (int m = 1; m <= n; ++m)
                for (int k = 1; k <= m; ++k) {
                    if (F[xp][m - k] == OR_INF || Vb[k] == OR_INF) continue;
                    uint64_t v = F[xp][m - k] > Vb[k] ? F[xp][m - k] : Vb[k];
                    if (v < F[x][m]) F[x][m] = v;
                }
        }
    uint64_t r = F[C][n];
    free(V);
    return r;
}

/* Step 2 tables for one band: Gs[y][k] = min Q for rows [y,R) in k slices. */
static void band_minsum(const dpctx_t *d, int x0, int x1, uint64_t Gs[OR_MAX_R + 1][OR_MAX_N + 1]) {
    const frame_t *f = d->f;
    int R = f->R, n = d->n;
    for (int y = 0; y <= R; ++y)
        for (int k = 0; k <= n; ++k) Gs[y][k] = OR_INF;
    Gs[R][0] = 0;
    for (int y = R - 1; y >= 0; --y)
        for (int y1 = y + 1; y1 <= R; ++y1) {
            rsum_t s = memo_get(d->memo, x0, x1, y, y1);
            if (!strip_ok(d, s, 2)) continue;
            uint64_t qs = sse_floor(s.S1, s.S2, s.N);
            for (int k = 1; k <= n; ++k) {
                if (Gs[y1][k - 1] == OR_INF) continue;
                uint64_t v = Gs[y1][k - 1] + qs;
                if (v < Gs[y][k]) Gs[y][k] = v;
            }
        }
}

/* Lex-smallest cut bits of a k-slice split of band [x0,x1) reaching Gs[0][k]. */
static uint64_t band_lexmin_bits(const dpctx_t *d, int x0, int x1,
                                 uint64_t Gs[OR_MAX_R + 1][OR_MAX_N + 1], int k) {
    const frame_t *f = d->f;
    int R = f->R;
    uint64_t bits = 0;
    int y = 0, kk = k;
    while (kk > 1) {
        /* the largest next cut keeps the bit string smallest */
        int chosen = -1;
        for (int y1 = R - 1; y1 > y; --y1) {
            rsum_t s = memo_get(d->memo, x0, x1, y, y1);
            if (!strip_ok(d, s, 2) || Gs[y1][kk - 1] == OR_INF) continue;
            if (Gs[y1][kk - 1] + sse_floor(s.S1, s.S2, s.N) == Gs[y][kk]) {
                chosen = y1;
                break;
            }
        }
        if (chosen < 0) return OR_INF; /* cannot happen when Gs[y][kk] is finite */
        bits |= 1ull << (chosen - 1);
        y = chosen;
        kk--;
    }
    return bits;
}

/* bit strings top to bottom with line 1 first: compare as reversed bit order */
static int bits_less(uint64_t a, uint64_t b, int R) {
    for (int y = 1; y < R; ++y) {
        int ba = (int)((a >> (y - 1)) & 1u), bb = (int)((b >> (y - 1)) & 1u);
        if (ba != bb) return ba < bb;
    }
    return 0;
}

typedef struct {
    int c;
    int x_edges[OR_MAX_C + 1];
    uint64_t band_cuts[OR_MAX_C];
    uint64_t q, t;
} code_t;

static int code_less(const code_t *a, const code_t *b, int R) {
    int c = a->c < b->c ? a->c : b->c;
    for (int i = 0; i < c; ++i) {
        if (a->x_edges[i + 1] != b->x_edges[i + 1]) return a->x_edges[i + 1] < b->x_edges[i + 1];
        if (a->band_cuts[i] != b->band_cuts[i]) return bits_less(a->band_cuts[i], b->band_cuts[i], R);
    }
    return 0;
}

/* Step 2 within one window: Q_w and its lex-smallest minimiser. */
static uint64_t window_step2(const dpctx_t *d, code_t *best) {
    const frame_t *f = d->f;
    int C = f->C, R = f->R, n = d->n;
    size_t nbands = (size_t)(C + 1) * (C + 1);
    uint64_t *V = (uint64_t *)malloc(sizeof(uint64_t) * nbands * (n + 1));
    uint64_t(*Gs)[OR_MAX_N + 1] = malloc(sizeof(uint64_t) * (OR_MAX_R + 1) * (OR_MAX_N + 1));
    if (!V || !Gs) {
        free(V);
        free(Gs);
        return OR_INF;
    }
    for (int x0 = 0; x0 < C; ++x0)
        for (int x1 = x0 + 1; x1 <= C; ++x1) {
            band_minsum(d, x0, x1, Gs);
            for (int k = 0; k <= n; ++k) V[((size_t)x0 * (C + 1) + x1) * (n + 1) + k] = Gs[0][k];
        }
    /* H[x][m]: columns [x,C) with m slices */
    uint64_t H[OR_MAX_C + 1][OR_MAX_N + 1];
    for (int x = 0; x <= C; ++x)
        for (int m = 0; m <= n; ++m) H[x][m] = OR_INF;
    H[C][0] = 0;
    for (int x = C - 1; x >= 0; --x)
        for (int x1 = x + 1; x1 <= C; ++x1) {
            const uint64_t *Vb = V + ((size_t)x * (C + 1) + x1) * (n + 1);
            for (int m = 1; m <= n; ++m)
                for (int k = 1; k <= m; ++k) {
                    if (Vb[k] == OR_INF || H[x1][m - k] == OR_INF) continue;
                    uint64_t v = Vb[k] + H[x1][m - k];
                    if (v < H[x][m]) H[x][m] = v;
                }
        }
    uint64_t qw = H[0][n];
    if (qw != OR_INF) {
        /* rebuild the lex-smallest code: smallest next edge, then smallest bits */
        int x = 0, m = n;
        best->c = 0;
        best->x_edges[0] = 0;
        best->q = qw;
        best->t = 0;
        while (x < C) {
            int found = 0;
            for (int x1 = x + 1; x1 <= C && !found; ++x1) {
                const uint64_t *Vb = V + ((size_t)x * (C + 1) + x1) * (n + 1);
                uint64_t bbits = 0;
                int bk = -1;
                int need_tables = 1;
                for (int k = 1; k <= m; ++k) {
                    if (Vb[k] == OR_INF || H[x1][m - k] == OR_INF) continue;
                    if (Vb[k] + H[x1][m - k] != H[x][m]) continue;
                    if (need_tables) {
                        band_minsum(d, x, x1, Gs);
                        need_tables = 0;
                    }
                    uint64_t bits = band_lexmin_bits(d, x, x1, Gs, k);
                    if (bk < 0 || bits_less(bits, bbits, R)) {
                        bbits = bits;
                        bk = k;
                    }
                }
                if (bk >= 0) {
                    best->band_cuts[best->c] = bbits;
                    best->c++;
                    best->x_edges[best->c] = x1;
                    x = x1;
                    m -= bk;
                    found = 1;
                }
            }
            if (!found) break; /* cannot happen when H[0][n] is finite */
        }
        /* T of the rebuilt partition */
        for (int b = 0; b < best->c; ++b) {
            int y0 = 0;
            for (int y = 1; y <= R; ++y)
                if (y == R || ((best->band_cuts[b] >> (y - 1)) & 1u)) {
                    rsum_t s = memo_get(d->memo, best->x_edges[b], best->x_edges[b + 1], y0, y);
                    if (s.T > best->t) best->t = s.T;
                    y0 = y;
                }
        }
    }
    free(V);
    free(Gs);
    return qw;
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* Distinct slice areas a with a*n <= A and (k*a-1)*n >= A: the windows that can hold a partition. */
static int list_windows(const frame_t *f, int n, int k_area, uint64_t **out, int *count) {
    int C = f->C, R = f->R;
    size_t cap = (size_t)C * (C + 1) / 2 * R * (R + 1) / 2;
    uint64_t *a = (uint64_t *)malloc(sizeof(uint64_t) * (cap ? cap : 1));
    if (!a) return OR_ENOMEM;
    size_t cnt = 0;
    uint64_t A = (uint64_t)f->W * f->H;
    for (int x0 = 0; x0 < C; ++x0)
        for (int x1 = x0 + 1; x1 <= C; ++x1)
            for (int y0 = 0; y0 < R; ++y0)
                for (int y1 = y0 + 1; y1 <= R; ++y1) {
                    uint64_t w = 0, h = 0;
                    for (int x = x0; x < x1; ++x) w += ctu_w(f, x);
                    for (int y = y0; y < y1; ++y) h += ctu_h(f, y);
                    uint64_t ar = w * h;
                    if (ar * (uint64_t)n <= A && ((uint64_t)k_area * ar - 1) * (uint64_t)n >= A) a[cnt++] = ar;
                }
    qsort(a, cnt, sizeof(uint64_t), cmp_u64);
    size_t u = 0;
    for (size_t i = 0; i < cnt; ++i)
        if (u == 0 || a[i] != a[u - 1]) a[u++] = a[i];
    *out = a;
    *count = (int)u;
    return OR_OK;
}

/*
 * O2.  Same result as O1 (area rule on) by facts (i) and (ii) above:
 * step 1 min over windows of the min-max DP; step 2 min over windows of the
 * min-sum DP under Eq. 4; ties to the lex-smallest code over all windows.
 */
static int search_dp_windows(int W, int H, const uint64_t *S1, const uint64_t *S2, const uint64_t *N,
                             const uint32_t *Tq, int n, int k_area, uint32_t lambda_q, int window_step,
                             oracle_result *res);

int oracle_search_dp(int W, int H, const uint64_t *S1, const uint64_t *S2, const uint64_t *N,
                     const uint32_t *Tq, int n, int k_area, uint32_t lambda_q, oracle_result *res) {
    return search_dp_windows(W, H, S1, S2, N, Tq, n, k_area, lambda_q, 1, res);
}

/*
 * Lightweight variant (the paper's future work on cheaper searches, Sec. 4):
 * the same DP over every window_step-th area window only, counted from the
 * largest window down (which always stays).  The result is a partition of
 * S(n) that is optimal among the partitions of those windows; step 1 is O2.
 */
int oracle_search_dp_windows(int W, int H, const uint64_t *S1, const uint64_t *S2, const uint64_t *N,
                             const uint32_t *Tq, int n, int k_area, uint32_t lambda_q, int window_step,
                             oracle_result *res) {
    return search_dp_windows(W, H, S1, S2, N, Tq, n, k_area, lambda_q, window_step, res);
}

static int search_dp_windows(int W, int H, const uint64_t *S1, const uint64_t *S2, const uint64_t *N,
                             const uint32_t *Tq, int n, int k_area, uint32_t lambda_q, int window_step,
                             oracle_result *res) {
    memset(res, 0, sizeof(*res));
    if (window_step < 1) {
        res->status = OR_EINVAL;
        return OR_EINVAL;
    }
    int st = check_inputs(W, H, n, k_area);
    if (st) {
        res->status = st;
        return st;
    }
    frame_t f = {W, H, (W + OR_CTU - 1) / OR_CTU, (H + OR_CTU - 1) / OR_CTU, S1, S2, N, Tq};
    memo_t m;
    if (memo_init(&m, &f)) {
        memo_free(&m);
        res->status = OR_ENOMEM;
        return OR_ENOMEM;
    }
    uint64_t *win = NULL;
    int nw = 0;
    if (list_windows(&f, n, k_area, &win, &nw)) {
        memo_free(&m);
        res->status = OR_ENOMEM;
        return OR_ENOMEM;
    }
    if (window_step > 1) { /* keep windows nw-1, nw-1-step, ... */
        int kept = 0;
        for (int i = 0; i < nw; ++i)
            if ((nw - 1 - i) % window_step == 0) win[kept++] = win[i];
        nw = kept;
    }
    res->n = n;
    res->n_windows = (uint64_t)nw;
    dpctx_t d = {&f, &m, n, k_area, 0, 0, 0};
    uint64_t t_min = OR_INF;
    for (int i = 0; i < nw; ++i) {
        d.a_lo = win[i];
        d.a_hi = (uint64_t)k_area * win[i] - 1;
        uint64_t t = window_tmin(&d);
        if (t < t_min) t_min = t;
    }
    if (t_min == OR_INF) {
        free(win);
        memo_free(&m);
        res->status = OR_EINFEASIBLE;
        return OR_EINFEASIBLE;
    }
    d.thr = eq4_thr(t_min, lambda_q);
    code_t best, cur;
    memset(&best, 0, sizeof(best));
    memset(&cur, 0, sizeof(cur));
    int have = 0;
    for (int i = 0; i < nw; ++i) {
        d.a_lo = win[i];
        d.a_hi = (uint64_t)k_area * win[i] - 1;
        uint64_t q = window_step2(&d, &cur);
        if (q == OR_INF) continue;
        if (!have || q < best.q || (q == best.q && code_less(&cur, &best, f.R))) {
            best = cur;
            have = 1;
        }
    }
    free(win);
    if (!have) { /* cannot happen: the T_min partition satisfies Eq. 4 */
        memo_free(&m);
        res->status = OR_EINFEASIBLE;
        return OR_EINFEASIBLE;
    }
    res->c = best.c;
    res->r = 1;
    res->row_mask = 0;
    for (int b = 0; b <= best.c; ++b) res->x_edges[b] = best.x_edges[b];
    for (int b = 0; b < best.c; ++b) res->band_cuts[b] = best.band_cuts[b];
    res->t_min = t_min;
    res->thr = d.thr;
    res->t = best.t;
    res->q = best.q;
    fill_reporting(&f, &m, res);
    memo_free(&m);
    res->status = OR_OK;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Multi-tile rectangular slices                                       */
/*
 * A wider reading of the slice shapes of Sec. 1 (Fig. 1b): a slice is either
 * a run of complete CTU rows inside one tile (as above) or a rectangle of
 * two or more complete tiles.  A configuration is a tile grid (column lines
 * X, row lines Y) whose tiles are grouped into rectangles of tiles; a group
 * of one tile holds k >= 1 in-tile slices, a larger group is one slice.
 * Exactly n slices, the area rule and the objective are as above.  Different
 * configurations can give the same slices; the search is over slice sets,
 * and ties on Q go to the smallest slice list in raster order (slices sorted
 * by top row, then left column, compared as (y0, x0, y1, x1)).
 *
 * Enumeration: row-line masks, then column-line masks, in increasing order;
 * the tiles grouped from the first ungrouped tile in raster order (width,
 * then height, increasing); a single tile's in-tile cuts as increasing masks.
 */
typedef struct {
    int status;
    int n;
    uint64_t t_min, thr, t, q;
    uint64_t n_sets;         /* distinct slice sets passing the area rule (count mode) */
    int16_t region[OR_MAX_N][4];   /* x0, y0, x1, y1 in CTUs, raster order */
    double sse_real;
} oracle_mt_result;

typedef struct {
    const frame_t *f;
    memo_t *m;
    int n, k_area, C, R;
    int xs[OR_MAX_C + 1], ys[OR_MAX_R + 1], c, r;
    int grp[OR_MAX_R][OR_MAX_C];     /* tile grouped? */
    int rect[OR_MAX_N][4];           /* x0, x1, y0, y1 of the slices so far */
    int ns;
    int mode;                        /* 0: step 1, 1: step 2, 2: collect keys */
    uint64_t t_min, thr;
    int have;
    uint64_t best_q, best_t;
    int best_key[OR_MAX_N][4];       /* y0, x0, y1, x1 in raster order */
    int16_t *keys;                   /* count mode: n*4 entries per slice set */
    size_t nkeys, capkeys;
    int oom;
    uint64_t n_sets;                 /* rectangle partitions visited (oracle_mt_search_rects) */
} mt_t;

static int key_cmp4(const int *a, const int *b) {
    for (int j = 0; j < 4; ++j)
        if (a[j] != b[j]) return a[j] < b[j] ? -1 : 1;
    return 0;
}

static void mt_evaluate(mt_t *e) {
    const frame_t *f = e->f;
    /* the slice list in raster order, as (y0, x0, y1, x1) */
    int key[OR_MAX_N][4];
    for (int i = 0; i < e->n; ++i) {
        key[i][0] = e->rect[i][2];
        key[i][1] = e->rect[i][0];
        key[i][2] = e->rect[i][3];
        key[i][3] = e->rect[i][1];
    }
    for (int i = 1; i < e->n; ++i)  /* insertion sort */
        for (int j = i; j > 0 && key_cmp4(key[j], key[j - 1]) < 0; --j)
            for (int q = 0; q < 4; ++q) {
                int t = key[j][q];
                key[j][q] = key[j - 1][q];
                key[j - 1][q] = t;
            }
    uint64_t amin = OR_INF, amax = 0, tmax = 0, qsum = 0;
    for (int i = 0; i < e->n; ++i) {
        rsum_t s = memo_get(e->m, key[i][1], key[i][3], key[i][0], key[i][2]);
        amin = s.N < amin ? s.N : amin;
        amax = s.N > amax ? s.N : amax;
        tmax = s.T > tmax ? s.T : tmax;
        qsum += sse_floor(s.S1, s.S2, s.N);
    }
    if (!((uint64_t)e->k_area * amin > amax)) return;
    if (e->mode == 2) {
        if (e->nkeys == e->capkeys) {
            size_t cap = e->capkeys ? 2 * e->capkeys : 1024;
            int16_t *k2 = (int16_t *)realloc(e->keys, cap * (size_t)e->n * 4 * sizeof(int16_t));
            if (!k2) {
                e->oom = 1;
                return;
            }
            e->keys = k2;
            e->capkeys = cap;
        }
        int16_t *dst = e->keys + e->nkeys * (size_t)e->n * 4;
        for (int i = 0; i < e->n; ++i)
            for (int q = 0; q < 4; ++q) dst[i * 4 + q] = (int16_t)key[i][q];
        e->nkeys++;
        return;
    }
    if (e->mode == 0) {
        if (tmax < e->t_min) e->t_min = tmax;
        return;
    }
    if (tmax > e->thr) return;
    int better = !e->have || qsum < e->best_q;
    if (!better && qsum == e->best_q)
        for (int i = 0; i < e->n; ++i) {
            int c = key_cmp4(key[i], e->best_key[i]);
            if (c) {
                better = c < 0;
                break;
            }
        }
    if (!better) return;
    e->have = 1;
    e->best_q = qsum;
    e->best_t = tmax;
    for (int i = 0; i < e->n; ++i)
        for (int q = 0; q < 4; ++q) e->best_key[i][q] = key[i][q];
    (void)f;
}

static void mt_group(mt_t *e);

/* in-tile cuts of a single tile [x0,x1) x [ty0,ty1): rows ty0+1 .. ty1-1 */
static void mt_split(mt_t *e, int x0, int x1, int ty0, int ty1) {
    const int h = ty1 - ty0;
    for (uint64_t cm = 0; cm < (1ull << (h - 1)); ++cm) {
        const int k = __builtin_popcountll(cm) + 1;
        if (e->ns + k > e->n) continue;
        int y0 = ty0;
        for (int y = ty0 + 1; y <= ty1; ++y) {
            if (y < ty1 && !((cm >> (y - ty0 - 1)) & 1ull)) continue;
            e->rect[e->ns][0] = x0;
            e->rect[e->ns][1] = x1;
            e->rect[e->ns][2] = y0;
            e->rect[e->ns][3] = y;
            e->ns++;
            y0 = y;
        }
        mt_group(e);
        e->ns -= k;
    }
}

static void mt_group(mt_t *e) {
    if (e->oom) return;
    int tx = -1, ty = -1;
    for (int j = 0; j < e->r && tx < 0; ++j)
        for (int i = 0; i < e->c; ++i)
            if (!e->grp[j][i]) {
                tx = i;
                ty = j;
                break;
            }
    if (tx < 0) {
        if (e->ns == e->n) mt_evaluate(e);
        return;
    }
    if (e->ns >= e->n) return;  /* an ungrouped tile still needs a slice */
    for (int w = 1; tx + w <= e->c && !e->grp[ty][tx + w - 1]; ++w)
        for (int h = 1; ty + h <= e->r; ++h) {
            int freecells = 1;
            for (int i = tx; i < tx + w && freecells; ++i)
                if (e->grp[ty + h - 1][i]) freecells = 0;
            if (!freecells) break;
            for (int j = ty; j < ty + h; ++j)
                for (int i = tx; i < tx + w; ++i) e->grp[j][i] = 1;
            if (w == 1 && h == 1) {
                mt_split(e, e->xs[tx], e->xs[tx + 1], e->ys[ty], e->ys[ty + 1]);
            } else {
                e->rect[e->ns][0] = e->xs[tx];
                e->rect[e->ns][1] = e->xs[tx + w];
                e->rect[e->ns][2] = e->ys[ty];
                e->rect[e->ns][3] = e->ys[ty + h];
                e->ns++;
                mt_group(e);
                e->ns--;
            }
            for (int j = ty; j < ty + h; ++j)
                for (int i = tx; i < tx + w; ++i) e->grp[j][i] = 0;
        }
}

static void mt_all(mt_t *e) {
    const int C = e->C, R = e->R;
    for (uint64_t ym = 0; ym < (1ull << (R - 1)); ++ym) {
        e->r = 0;
        e->ys[0] = 0;
        for (int y = 1; y < R; ++y)
            if ((ym >> (y - 1)) & 1ull) e->ys[++e->r] = y;
        e->ys[++e->r] = R;
        for (uint64_t xm = 0; xm < (1ull << (C - 1)); ++xm) {
            e->c = 0;
            e->xs[0] = 0;
            for (int x = 1; x < C; ++x)
                if ((xm >> (x - 1)) & 1ull) e->xs[++e->c] = x;
            e->xs[++e->c] = C;
            memset(e->grp, 0, sizeof(e->grp));
            e->ns = 0;
            mt_group(e);
        }
    }
}

static int cmp_keys_n;
static int cmp_keys(const void *a, const void *b) {
    const int16_t *x = (const int16_t *)a, *y = (const int16_t *)b;
    for (int i = 0; i < cmp_keys_n * 4; ++i)
        if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
    return 0;
}

/* Shapes with up to 16 column and 16 row lines only: the enumeration is exponential in both. */
static int mt_setup(mt_t *e, frame_t *f, memo_t *m, int W, int H, int n, int k_area) {
    int st = check_inputs(W, H, n, k_area);
    if (st) return st;
    memset(e, 0, sizeof(*e));
    e->f = f;
    e->m = m;
    e->n = n;
    e->k_area = k_area;
    e->C = f->C;
    e->R = f->R;
    if (f->C > 17 || f->R > 17) return OR_EINVAL;
    return OR_OK;
}

int oracle_mt_count(int W, int H, int n, int k_area, uint64_t *count) {
    if (!count) return OR_EINVAL;
    const int C = (W + OR_CTU - 1) / OR_CTU, R = (H + OR_CTU - 1) / OR_CTU;
    size_t cells = (size_t)(C > 0 ? C : 1) * (R > 0 ? R : 1);
    uint64_t *ones = (uint64_t *)calloc(cells, sizeof(uint64_t));
    uint32_t *zeros = (uint32_t *)calloc(cells, sizeof(uint32_t));
    if (!ones || !zeros) {
        free(ones);
        free(zeros);
        return OR_ENOMEM;
    }
    frame_t f = {W, H, C, R, ones, ones, NULL, zeros};
    uint64_t *N = (uint64_t *)calloc(cells, sizeof(uint64_t));
    if (!N) {
        free(ones);
        free(zeros);
        return OR_ENOMEM;
    }
    for (int y = 0; y < R; ++y)
        for (int x = 0; x < C; ++x) N[y * C + x] = (uint64_t)ctu_w(&f, x) * ctu_h(&f, y);
    f.N = N;
    memo_t m;
    mt_t e;
    int st = OR_ENOMEM;
    if (!memo_init(&m, &f)) {
        st = mt_setup(&e, &f, &m, W, H, n, k_area);
        if (st == OR_OK) {
            e.mode = 2;
            mt_all(&e);
            if (e.oom) {
                st = OR_ENOMEM;
            } else {
                cmp_keys_n = n;
                qsort(e.keys, e.nkeys, (size_t)n * 4 * sizeof(int16_t), cmp_keys);
                uint64_t distinct = 0;
                for (size_t i = 0; i < e.nkeys; ++i)
                    if (i == 0 || cmp_keys(e.keys + (i - 1) * (size_t)n * 4, e.keys + i * (size_t)n * 4)) distinct++;
                *count = distinct;
            }
            free(e.keys);
        }
    }
    memo_free(&m);
    free(ones);
    free(zeros);
    free(N);
    return st;
}

int oracle_mt_search(int W, int H, const uint64_t *S1, const uint64_t *S2, const uint64_t *N, const uint32_t *Tq,
                     int n, int k_area, uint32_t lambda_q, oracle_mt_result *res) {
    memset(res, 0, sizeof(*res));
    frame_t f = {W, H, (W + OR_CTU - 1) / OR_CTU, (H + OR_CTU - 1) / OR_CTU, S1, S2, N, Tq};
    memo_t m;
    if (memo_init(&m, &f)) {
        memo_free(&m);
        res->status = OR_ENOMEM;
        return OR_ENOMEM;
    }
    mt_t e;
    int st = mt_setup(&e, &f, &m, W, H, n, k_area);
    if (st) {
        memo_free(&m);
        res->status = st;
        return st;
    }
    e.mode = 0;
    e.t_min = OR_INF;
    mt_all(&e);
    res->n = n;
    if (e.t_min == OR_INF) {
        memo_free(&m);
        res->status = OR_EINFEASIBLE;
        return OR_EINFEASIBLE;
    }
    e.thr = eq4_thr(e.t_min, lambda_q);
    e.mode = 1;
    mt_all(&e);
    res->t_min = e.t_min;
    res->thr = e.thr;
    res->t = e.best_t;
    res->q = e.best_q;
    long double sse = 0.0L;
    for (int i = 0; i < n; ++i) {
        res->region[i][0] = (int16_t)e.best_key[i][1];
        res->region[i][1] = (int16_t)e.best_key[i][0];
        res->region[i][2] = (int16_t)e.best_key[i][3];
        res->region[i][3] = (int16_t)e.best_key[i][2];
        rsum_t s = memo_get(&m, e.best_key[i][1], e.best_key[i][3], e.best_key[i][0], e.best_key[i][2]);
        sse += sse_exact(s.S1, s.S2, s.N);
    }
    res->sse_real = (double)sse;
    memo_free(&m);
    res->status = OR_OK;
    return OR_OK;
}

size_t oracle_mt_result_size(void) { return sizeof(oracle_mt_result); }

/* Objective of a given partition by direct sums (used to check any result). */
int oracle_evaluate(int W, int H, const uint64_t *S1, const uint64_t *S2, const uint64_t *N,
                    const uint32_t *Tq, int c, const int *x_edges, const uint64_t *band_cuts,
                    uint64_t *t_out, uint64_t *q_out, uint64_t *amin_out, uint64_t *amax_out,
                    int *nreg_out) {
    if (W <= 0 || H <= 0) return OR_EINVAL;
    frame_t f = {W, H, (W + OR_CTU - 1) / OR_CTU, (H + OR_CTU - 1) / OR_CTU, S1, S2, N, Tq};
    if (c < 1 || c > f.C || x_edges[0] != 0 || x_edges[c] != f.C) return OR_EINVAL;
    uint64_t t = 0, q = 0, amin = OR_INF, amax = 0;
    int nreg = 0;
    for (int b = 0; b < c; ++b) {
        if (x_edges[b + 1] <= x_edges[b]) return OR_EINVAL;
        int y0 = 0;
        for (int y = 1; y <= f.R; ++y)
            if (y == f.R || ((band_cuts[b] >> (y - 1)) & 1u)) {
                rsum_t s = rect_direct(&f, x_edges[b], x_edges[b + 1], y0, y);
                if (s.T > t) t = s.T;
                q += sse_floor(s.S1, s.S2, s.N);
                if (s.N < amin) amin = s.N;
                if (s.N > amax) amax = s.N;
                nreg++;
                y0 = y;
            }
    }
    *t_out = t;
    *q_out = q;
    *amin_out = amin;
    *amax_out = amax;
    *nreg_out = nreg;
    return OR_OK;
}

/* Time (Eq. 1) and floored SSE (Eq. 2) of one rectangle [x0,x1) x [y0,y1) by direct sums. */
int oracle_rect(int W, int H, const uint64_t *S1, const uint64_t *S2, const uint64_t *N, const uint32_t *Tq,
                int x0, int x1, int y0, int y1, uint64_t *t_out, uint64_t *q_out) {
    frame_t f = {W, H, (W + OR_CTU - 1) / OR_CTU, (H + OR_CTU - 1) / OR_CTU, S1, S2, N, Tq};
    if (x0 < 0 || x1 > f.C || x0 >= x1 || y0 < 0 || y1 > f.R || y0 >= y1) return OR_EINVAL;
    rsum_t s = rect_direct(&f, x0, x1, y0, y1);
    *t_out = s.T;
    *q_out = sse_floor(s.S1, s.S2, s.N);
    return OR_OK;
}

/* Time and floor SSE of every CTU rectangle, each by direct sums like
   oracle_rect: entry ((x0*(C+1) + x1)*(R+1) + y0)*(R+1) + y1 for x0 < x1,
   y0 < y1; the other entries are set to zero. */
int oracle_rect_all(int W, int H, const uint64_t *S1, const uint64_t *S2, const uint64_t *N, const uint32_t *Tq,
                    uint64_t *t_out, uint64_t *q_out) {
    if (W <= 0 || H <= 0) return OR_EINVAL;
    frame_t f = {W, H, (W + OR_CTU - 1) / OR_CTU, (H + OR_CTU - 1) / OR_CTU, S1, S2, N, Tq};
    if (f.C > OR_MAX_C || f.R > OR_MAX_R) return OR_EINVAL;
    size_t cells = (size_t)(f.C + 1) * (f.C + 1) * (f.R + 1) * (f.R + 1);
    memset(t_out, 0, cells * sizeof(uint64_t));
    memset(q_out, 0, cells * sizeof(uint64_t));
    for (int x0 = 0; x0 < f.C; ++x0)
        for (int x1 = x0 + 1; x1 <= f.C; ++x1)
            for (int y0 = 0; y0 < f.R; ++y0)
                for (int y1 = y0 + 1; y1 <= f.R; ++y1) {
                    size_t i = (((size_t)x0 * (f.C + 1) + x1) * (f.R + 1) + y0) * (f.R + 1) + y1;
                    rsum_t r = rect_direct(&f, x0, x1, y0, y1);
                    t_out[i] = r.T;
                    q_out[i] = sse_floor(r.S1, r.S2, r.N);
                }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* The multi-tile space again, as the partitions of the CTU grid into n
   rectangles (a grid with a line at every slice edge makes each rectangle a
   group of whole tiles, so this is the same set of slice sets as
   oracle_mt_search enumerates through tile grids; the tests check both
   against each other).  Reaches full frame sizes for small n.

   Every partition is made once: the first free CTU in raster order is the
   top-left corner of the next rectangle, whose width and then height grow.
   A partial set is not extended once its areas break k*A_min > A_max, or
   once the rest of the frame cannot be cut into the remaining rectangles
   under the rule (each of them needs an area s with k*s > A_max and
   s < k*A_min of the rectangles so far); no completion of it is valid. */

static uint64_t mtr_px(int i, int cells, int extent) {
    int e = i * OR_CTU;
    (void)cells;
    return (uint64_t)(e < extent ? e : extent);
}

static void mtr_rec(mt_t *e, uint64_t *freem, uint64_t rest, uint64_t amin, uint64_t amax) {
    const frame_t *f = e->f;
    int y = 0;
    while (y < f->R && freem[y] == 0) ++y;
    int left = e->n - e->ns;
    if (y == f->R) {
        if (left == 0) {
            if (e->mode == 0) e->n_sets++;
            mt_evaluate(e);
        }
        return;
    }
    if (left == 0) return;
    if (e->ns > 0 && !((u128)e->k_area * rest > (u128)left * amax &&
                       (u128)rest < (u128)left * (u128)e->k_area * amin))
        return;
    int x = 0;
    while (!((freem[y] >> x) & 1u)) ++x;
    for (int x1 = x + 1; x1 <= f->C && ((freem[y] >> (x1 - 1)) & 1u); ++x1) {
        uint64_t bits = (x1 == 64 ? ~0ull : ((1ull << x1) - 1)) & ~((1ull << x) - 1);
        for (int y1 = y + 1; y1 <= f->R && (freem[y1 - 1] & bits) == bits; ++y1) {
            uint64_t a = (mtr_px(x1, f->C, f->W) - mtr_px(x, f->C, f->W)) *
                         (mtr_px(y1, f->R, f->H) - mtr_px(y, f->R, f->H));
            uint64_t lo = a < amin ? a : amin, hi = a > amax ? a : amax;
            if (!((u128)e->k_area * lo > (u128)hi)) continue;
            for (int yy = y; yy < y1; ++yy) freem[yy] ^= bits;
            e->rect[e->ns][0] = x;
            e->rect[e->ns][1] = x1;
            e->rect[e->ns][2] = y;
            e->rect[e->ns][3] = y1;
            e->ns++;
            mtr_rec(e, freem, rest - a, lo, hi);
            e->ns--;
            for (int yy = y; yy < y1; ++yy) freem[yy] ^= bits;
        }
    }
}

static void mtr_all(mt_t *e) {
    const frame_t *f = e->f;
    uint64_t freem[OR_MAX_R];
    for (int y = 0; y < f->R; ++y) freem[y] = f->C == 64 ? ~0ull : ((1ull << f->C) - 1);
    e->ns = 0;
    mtr_rec(e, freem, (uint64_t)f->W * (uint64_t)f->H, OR_INF, 0);
}

/* The multi-tile search over the rectangle partitions: T_min (Eq. 3), then
   the smallest (Q, raster-ordered slice list) under Eq. 4, as
   oracle_mt_search; res->n_sets is the number of slice sets. */
int oracle_mt_search_rects(int W, int H, const uint64_t *S1, const uint64_t *S2, const uint64_t *N,
                           const uint32_t *Tq, int n, int k_area, uint32_t lambda_q, oracle_mt_result *res) {
    memset(res, 0, sizeof(*res));
    frame_t f = {W, H, (W + OR_CTU - 1) / OR_CTU, (H + OR_CTU - 1) / OR_CTU, S1, S2, N, Tq};
    memo_t m;
    if (memo_init(&m, &f)) {
        memo_free(&m);
        res->status = OR_ENOMEM;
        return OR_ENOMEM;
    }
    mt_t e;
    int st = check_inputs(W, H, n, k_area);
    if (st) {
        memo_free(&m);
        res->status = st;
        return st;
    }
    memset(&e, 0, sizeof(e));
    e.f = &f;
    e.m = &m;
    e.n = n;
    e.k_area = k_area;
    e.C = f.C;
    e.R = f.R;
    e.mode = 0;
    e.t_min = OR_INF;
    mtr_all(&e);
    res->n = n;
    res->n_sets = e.n_sets;
    if (e.t_min == OR_INF) {
        memo_free(&m);
        res->status = OR_EINFEASIBLE;
        return OR_EINFEASIBLE;
    }
    e.thr = eq4_thr(e.t_min, lambda_q);
    e.mode = 1;
    mtr_all(&e);
    res->t_min = e.t_min;
    res->thr = e.thr;
    res->t = e.best_t;
    res->q = e.best_q;
    long double sse = 0.0L;
    for (int i = 0; i < n; ++i) {
        res->region[i][0] = (int16_t)e.best_key[i][1];
        res->region[i][1] = (int16_t)e.best_key[i][0];
        res->region[i][2] = (int16_t)e.best_key[i][3];
        res->region[i][3] = (int16_t)e.best_key[i][2];
        rsum_t s = memo_get(&m, e.best_key[i][1], e.best_key[i][3], e.best_key[i][0], e.best_key[i][2]);
        sse += sse_exact(s.S1, s.S2, s.N);
    }
    res->sse_real = (double)sse;
    memo_free(&m);
    res->status = OR_OK;
    return OR_OK;
}

size_t oracle_result_size(void) { return sizeof(oracle_result); }
