/*
 * svf_oracle.c -- plain, slow, FP64 CPU oracle for the SVFusion hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the package's smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no source,
 * header, table or helper with the CUDA path; it is built by gcc with
 * -O2 -ffp-contract=off (no fused multiply-add, no fast-math) and is
 * parallel only across independent queries / vertices (OpenMP).
 *
 * What it computes, and where the paper defines it (SVFusion, arXiv
 * 2601.08528):
 *   orc_knn          exact k nearest neighbours by (distance, id)   Sec. 2.1
 *   orc_search       Algorithm 1 on the GPU-resident graph: random
 *                    candidate-pool initialisation, repeat {nearest
 *                    unexpanded entry, fetch its neighbours, distances,
 *                    update the size-L pool}; top-k        Alg. 1, Sec. 4.2
 *   orc_prune        neighbour reordering of a sorted candidate list:
 *                    detour counts, stable ascending sort, first R; the
 *                    rank-based count of Sec. 5.1 and a distance-based
 *                    (relative-neighbourhood) count               Sec. 5.1
 *   orc_build        exact 2R-NN graph, each row pruned to R       Sec. 3, 4.2
 *   orc_insert       search for candidates, prune, forward row,
 *                    reverse-edge patch                            Sec. 5.1
 *   orc_delete       logical delete in a bitset + localized repair of
 *                    vertices with > 50% deleted out-neighbours
 *                    using at most c entries of each deleted
 *                    neighbour's list                              Sec. 5.2
 *   codecs           bfloat16 (round to nearest even) and OCP FP8 E4M3FN
 *                    (satfinite) written from the format definitions.
 *   MLP              16-64-1 stop predictor forward/backward (FP64).
 *
 * Readings where the paper is silent (they are the same on the GPU side):
 *   - the loop runs a fixed number T of iterations; an iteration with no
 *     unexpanded pool entry changes nothing (Alg. 1 "until unchanged");
 *   - "GetNearest" is the nearest *unexpanded* entry, one per iteration;
 *   - every order is lexicographic (distance, id); detour tests are strict;
 *   - L2 is squared Euclidean; inner product is scored as -<q,x>;
 *   - random initialisation draws id_j = floor(hi32(splitmix64(base ^ j)) *
 *     n_used / 2^32) (the multiply-shift range reduction of Lemire, 2019),
 *     base = splitmix64(seed ^ splitmix64(qkey)), j = 0,1,..., keeping the
 *     first L distinct live ids within 4L draws; qkey is the caller's key or
 *     the wrapping sum over the query's little-endian 32-bit words w_i of
 *     splitmix64((i << 32) | w_i).
 *
 * Parity support: every function that orders floating-point distances also
 * reports the smallest *relative gap* among the comparisons that decided its
 * result (pool truncation, parent choice, output order, kNN boundary, detour
 * tests).  A GPU result computed in FP32 may legitimately differ from this
 * FP64 one only where such a gap is tiny.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_EMPTY 0xFFFFFFFFu
#define ORC_MAX_W 32 /* most parents per iteration */

enum { ORC_F32 = 0, ORC_U8 = 1, ORC_BF16 = 2, ORC_FP8 = 3 };
enum { ORC_L2 = 0, ORC_IP = 1 };
enum { ORC_PRUNE_RNG = 0, ORC_PRUNE_RANK = 1 };

typedef struct {
    const void *data; /* row-major rows, `pitch` bytes apart */
    int64_t n;        /* rows present */
    int32_t d;        /* dimension */
    int32_t dtype;    /* ORC_F32 / ORC_U8 / ORC_BF16 / ORC_FP8 */
    int64_t pitch;    /* bytes between rows; FP8 keeps its fp32 scale at byte d */
    int32_t metric;   /* ORC_L2 / ORC_IP */
    int32_t pad_;
} orc_store;

/* ------------------------------------------------------------------ */
/* splitmix64 (Steele, Lea, Flood 2014; constants as published by Vigna) */
static uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64(uint64_t x) { return splitmix64(x); }

/* Key of a query from its raw bytes (nbytes a multiple of 4). */
uint64_t orc_query_key(const void *q, int64_t nbytes) {
    const uint8_t *b = (const uint8_t *)q;
    uint64_t h = 0;
    for (int64_t i = 0; i < nbytes / 4; i++) {
        uint32_t w = (uint32_t)b[4 * i] | ((uint32_t)b[4 * i + 1] << 8) |
                     ((uint32_t)b[4 * i + 2] << 16) | ((uint32_t)b[4 * i + 3] << 24);
        h += splitmix64(((uint64_t)i << 32) | w);
    }
    return h;
}

/* ------------------------------------------------------------------ */
/* Codecs from their format definitions.                              */

/* bfloat16: the upper 16 bits of an IEEE binary32, rounded to nearest,
   ties to even.  NaN stays a (quiet) NaN. */
uint16_t orc_bf16_encode(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu))
        return (uint16_t)((u >> 16) | 0x0040u);
    uint32_t hi = u >> 16, lo = u & 0xFFFFu;
    if (lo > 0x8000u || (lo == 0x8000u && (hi & 1u)))
        hi += 1; /* carry into the exponent is the correct overflow to inf */
    return (uint16_t)hi;
}

double orc_bf16_decode(uint16_t h) {
    uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

/* OCP 8-bit floating point, E4M3FN: 1 sign, 4 exponent (bias 7), 3 mantissa
   bits; no infinities; S.1111.111 is NaN; largest finite 448. */
double orc_e4m3_decode(uint8_t c) {
    int s = c >> 7, e = (c >> 3) & 15, m = c & 7;
    double v;
    if (e == 15 && m == 7)
        return NAN;
    if (e == 0)
        v = ldexp((double)m, -9); /* subnormal: m/8 * 2^-6 */
    else
        v = ldexp(1.0 + m / 8.0, e - 7);
    return s ? -v : v;
}

/* Round-to-nearest-even encode with saturation to +-448 (satfinite). */
uint8_t orc_e4m3_encode(float xf) {
    double x = (double)xf;
    if (isnan(x))
        return 0x7F;
    uint8_t sign = signbit(x) ? 0x80 : 0;
    double a = fabs(x);
    if (a >= 448.0)
        return sign | 0x7E;
    int e;
    (void)frexp(a, &e); /* a = f * 2^e, f in [0.5, 1) */
    e -= 1;             /* a = mant * 2^e, mant in [1, 2) */
    if (a == 0.0 || e < -6) {
        double q = nearbyint(ldexp(a, 9)); /* units of 2^-9 */
        return sign | (uint8_t)q;           /* q == 8 is exactly the smallest normal */
    }
    double m = nearbyint((ldexp(a, -e) - 1.0) * 8.0);
    if (m == 8.0) {
        m = 0.0;
        e += 1;
    }
    int code = ((e + 7) << 3) | (int)m;
    if (code > 0x7E)
        code = 0x7E;
    return sign | (uint8_t)code;
}

/* Per-vector scaled FP8 rows: s = max|x| / 448 (1 if x == 0), code_i =
   E4M3(x_i / s) with both divisions rounded to binary32; s stored as fp32 at
   byte offset d of the row. */
void orc_fp8_encode_rows(const float *x, int64_t n, int32_t d, uint8_t *out, int64_t pitch) {
    for (int64_t r = 0; r < n; r++) {
        const float *xr = x + r * d;
        uint8_t *o = out + r * pitch;
        float mx = 0.0f;
        for (int i = 0; i < d; i++) {
            float a = fabsf(xr[i]);
            if (a > mx)
                mx = a;
        }
        volatile float s = (mx == 0.0f) ? 1.0f : mx / 448.0f;
        for (int i = 0; i < d; i++) {
            volatile float v = xr[i] / s;
            o[i] = orc_e4m3_encode(v);
        }
        float sv = s;
        memcpy(o + d, &sv, 4);
    }
}

void orc_bf16_encode_rows(const float *x, int64_t n, int32_t d, uint16_t *out, int64_t pitch_bytes) {
    for (int64_t r = 0; r < n; r++)
        for (int i = 0; i < d; i++)
            *(uint16_t *)((uint8_t *)out + r * pitch_bytes + 2 * i) = orc_bf16_encode(x[r * d + i]);
}

/* ------------------------------------------------------------------ */
/* Distances in FP64.                                                 */

static void decode_row(const orc_store *X, int64_t id, double *out) {
    const uint8_t *row = (const uint8_t *)X->data + id * X->pitch;
    int d = X->d;
    switch (X->dtype) {
    case ORC_F32:
        for (int i = 0; i < d; i++) {
            float f;
            memcpy(&f, row + 4 * i, 4);
            out[i] = f;
        }
        break;
    case ORC_U8:
        for (int i = 0; i < d; i++)
            out[i] = row[i];
        break;
    case ORC_BF16:
        for (int i = 0; i < d; i++) {
            uint16_t h;
            memcpy(&h, row + 2 * i, 2);
            out[i] = orc_bf16_decode(h);
        }
        break;
    default: { /* FP8 */
        float s;
        memcpy(&s, row + d, 4);
        for (int i = 0; i < d; i++)
            out[i] = orc_e4m3_decode(row[i]) * (double)s;
    }
    }
}

/* The query as doubles: u8 queries for a u8 store, fp32 otherwise. */
static void decode_query(const orc_store *X, const void *Q, int64_t qi, double *out) {
    int d = X->d;
    if (X->dtype == ORC_U8) {
        const uint8_t *q = (const uint8_t *)Q + qi * d;
        for (int i = 0; i < d; i++)
            out[i] = q[i];
    } else {
        const float *q = (const float *)Q + qi * d;
        for (int i = 0; i < d; i++)
            out[i] = q[i];
    }
}

static int64_t query_bytes(const orc_store *X) { return (int64_t)X->d * (X->dtype == ORC_U8 ? 1 : 4); }

/* dist(a, b) and its magnitude scale (|dist| for L2, sum |a_i b_i| for IP),
   the denominator of a relative gap.  For integer inputs every term is an
   exact integer below 2^53, so the result is exact. */
static double vdist(const double *a, const double *b, int d, int metric, double *scale) {
    double s = 0.0, t = 0.0;
    if (metric == ORC_L2) {
        for (int i = 0; i < d; i++) {
            double df = a[i] - b[i];
            s += df * df;
        }
        *scale = s;
        return s;
    }
    for (int i = 0; i < d; i++) {
        s += a[i] * b[i];
        t += fabs(a[i] * b[i]);
    }
    *scale = t;
    return -s;
}

static double rel_gap(double da, double sa, double db, double sb) {
    double den = sa > sb ? sa : sb;
    double g = fabs(da - db);
    if (den <= 0.0)
        return g > 0.0 ? INFINITY : 0.0;
    return g / den;
}

static int is_deleted(const uint32_t *del, uint32_t id) {
    return del && ((del[id >> 5] >> (id & 31)) & 1u);
}

/* ------------------------------------------------------------------ */
typedef struct {
    double d, s;  /* distance, magnitude scale */
    uint32_t id;
    int exp;      /* expanded flag (search pool only) */
} ent;

static int ent_cmp(const void *pa, const void *pb) {
    const ent *a = (const ent *)pa, *b = (const ent *)pb;
    if (a->d < b->d) return -1;
    if (a->d > b->d) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

/* An exact set of uint32 ids: open addressing with doubling. */
typedef struct {
    uint32_t *slot;
    int64_t cap, cnt;
} idset;

static void set_init(idset *s, int64_t cap) {
    s->cap = 64;
    while (s->cap < 2 * cap) s->cap <<= 1;
    s->slot = (uint32_t *)malloc(sizeof(uint32_t) * s->cap);
    memset(s->slot, 0xFF, sizeof(uint32_t) * s->cap);
    s->cnt = 0;
}
static void set_free(idset *s) { free(s->slot); }
static int set_has(const idset *s, uint32_t id) {
    uint64_t h = splitmix64(id) & (uint64_t)(s->cap - 1);
    while (s->slot[h] != ORC_EMPTY) {
        if (s->slot[h] == id) return 1;
        h = (h + 1) & (uint64_t)(s->cap - 1);
    }
    return 0;
}
static void set_add(idset *s, uint32_t id);
static void set_grow(idset *s) {
    idset t;
    t.cap = s->cap * 2;
    t.slot = (uint32_t *)malloc(sizeof(uint32_t) * t.cap);
    memset(t.slot, 0xFF, sizeof(uint32_t) * t.cap);
    t.cnt = 0;
    for (int64_t i = 0; i < s->cap; i++)
        if (s->slot[i] != ORC_EMPTY) set_add(&t, s->slot[i]);
    free(s->slot);
    *s = t;
}
static void set_add(idset *s, uint32_t id) {
    if (2 * (s->cnt + 1) > s->cap) set_grow(s);
    uint64_t h = splitmix64(id) & (uint64_t)(s->cap - 1);
    while (s->slot[h] != ORC_EMPTY) {
        if (s->slot[h] == id) return;
        h = (h + 1) & (uint64_t)(s->cap - 1);
    }
    s->slot[h] = id;
    s->cnt++;
}

/* ------------------------------------------------------------------ */
/* Exact kNN (Sec. 2.1): for each query, the k rows with the smallest
   (dist, id) among live rows [0, n), skipping row self_ids[qi] if given.
   out_gap[qi] (optional): the smallest relative gap between consecutive
   entries of the first k+1 (the k-boundary and the output order). */
void orc_knn(const orc_store *X, const uint32_t *del, const void *Q, int64_t nq,
             const int64_t *self_ids, int32_t k, uint32_t *out_ids, double *out_d, double *out_gap) {
    int d = X->d;
#pragma omp parallel
    {
        double *q = (double *)malloc(sizeof(double) * d);
        double *x = (double *)malloc(sizeof(double) * d);
        ent *best = (ent *)malloc(sizeof(ent) * (k + 2));
#pragma omp for schedule(dynamic, 4)
        for (int64_t qi = 0; qi < nq; qi++) {
            decode_query(X, Q, qi, q);
            int cnt = 0; /* best[] sorted, holds up to k+1 entries */
            for (int64_t id = 0; id < X->n; id++) {
                if (self_ids && self_ids[qi] == id) continue;
                if (is_deleted(del, (uint32_t)id)) continue;
                decode_row(X, id, x);
                ent e;
                e.d = vdist(q, x, d, X->metric, &e.s);
                e.id = (uint32_t)id;
                e.exp = 0;
                if (cnt == k + 1 && ent_cmp(&e, &best[k]) >= 0) continue;
                int pos = cnt < k + 1 ? cnt++ : k;
                while (pos > 0 && ent_cmp(&e, &best[pos - 1]) < 0) {
                    best[pos] = best[pos - 1];
                    pos--;
                }
                best[pos] = e;
            }
            double g = INFINITY;
            for (int i = 0; i + 1 < cnt; i++) {
                double gi = rel_gap(best[i].d, best[i].s, best[i + 1].d, best[i + 1].s);
                if (gi < g) g = gi;
            }
            for (int i = 0; i < k; i++) {
                out_ids[qi * k + i] = i < cnt ? best[i].id : ORC_EMPTY;
                if (out_d) out_d[qi * k + i] = i < cnt ? best[i].d : INFINITY;
            }
            if (out_gap) out_gap[qi] = g;
        }
        free(q);
        free(x);
        free(best);
    }
}

/* ------------------------------------------------------------------ */
/* Neighbour reordering (Sec. 5.1).  `c` holds m candidates of vertex v,
   sorted by (dist, id).  count_i is
     RNG : #{ j < i : dist(c_j, c_i) < dist(v, c_i) }   (a shorter detour)
     RANK: #{ j < i : c_i is in N_out(c_j) }             (a detour edge)
   The candidates are stably sorted by ascending count and the first
   min(R, m) are written to out[] (the rest EMPTY).  For RANK, N_out(u) is
   row u of `nbr` (width nbr_w).  Returns the smallest relative gap of the
   RNG detour tests (INFINITY for RANK). */
static double prune_core(const orc_store *X, const ent *c, int m, int mode, const uint32_t *nbr,
                         int nbr_w, int R, uint32_t *out, double *xa, double *xb) {
    int *cnt = (int *)calloc((size_t)(m > 0 ? m : 1), sizeof(int));
    int *ord = (int *)malloc(sizeof(int) * (m > 0 ? m : 1));
    double g = INFINITY;
    for (int i = 0; i < m; i++) {
        if (mode == ORC_PRUNE_RNG) decode_row(X, c[i].id, xa);
        for (int j = 0; j < i; j++) {
            if (mode == ORC_PRUNE_RNG) {
                double s;
                decode_row(X, c[j].id, xb);
                double djk = vdist(xb, xa, X->d, X->metric, &s);
                if (djk < c[i].d) cnt[i]++;
                double gi = rel_gap(djk, s, c[i].d, c[i].s);
                if (gi < g) g = gi;
            } else {
                const uint32_t *row = nbr + (int64_t)c[j].id * nbr_w;
                for (int r = 0; r < nbr_w; r++)
                    if (row[r] == c[i].id) {
                        cnt[i]++;
                        break;
                    }
            }
        }
    }
    /* stable sort by count: insertion sort keeps equal counts in rank order */
    for (int i = 0; i < m; i++) {
        int p = i;
        while (p > 0 && cnt[ord[p - 1]] > cnt[i]) {
            ord[p] = ord[p - 1];
            p--;
        }
        ord[p] = i;
    }
    for (int r = 0; r < R; r++) out[r] = r < m ? c[ord[r]].id : ORC_EMPTY;
    free(cnt);
    free(ord);
    return g;
}

/* Public wrapper: candidates given as ids with their distances to v and
   magnitude scales (dist used for the RNG test). */
double orc_prune(const orc_store *X, const uint32_t *cand_ids, const double *cand_d, const double *cand_s,
                 int32_t m, int32_t mode, const uint32_t *nbr, int32_t nbr_w, int32_t R, uint32_t *out) {
    ent *c = (ent *)malloc(sizeof(ent) * (m > 0 ? m : 1));
    for (int i = 0; i < m; i++) {
        c[i].id = cand_ids[i];
        c[i].d = cand_d[i];
        c[i].s = cand_s ? cand_s[i] : fabs(cand_d[i]);
        c[i].exp = 0;
    }
    double *xa = (double *)malloc(sizeof(double) * X->d);
    double *xb = (double *)malloc(sizeof(double) * X->d);
    double g = prune_core(X, c, m, mode, nbr, nbr_w, R, out, xa, xb);
    free(xa);
    free(xb);
    free(c);
    return g;
}

/* ------------------------------------------------------------------ */
/* Build (Sec. 3 "Build", Sec. 4.2 "Index Construction"): the exact 2R
   nearest neighbours of every vertex (self excluded) by (dist, id), each
   list pruned to R.  rows_gap[v]: smallest relative gap of the kNN order
   and boundary and of the detour tests that decided row v. */
void orc_build(const orc_store *X, int32_t R, int32_t mode, uint32_t *graph, double *rows_gap) {
    int64_t n = X->n;
    int K = 2 * R;
    if (K > n - 1) K = (int)(n - 1);
    int d = X->d;
    uint32_t *knn = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n * (K > 0 ? K : 1));
    double *knd = (double *)malloc(sizeof(double) * (size_t)n * (K > 0 ? K : 1));
    double *kns = (double *)malloc(sizeof(double) * (size_t)n * (K > 0 ? K : 1));
    double *kgap = (double *)malloc(sizeof(double) * n);
#pragma omp parallel
    {
        double *q = (double *)malloc(sizeof(double) * d);
        double *x = (double *)malloc(sizeof(double) * d);
        ent *best = (ent *)malloc(sizeof(ent) * (K + 2));
#pragma omp for schedule(dynamic, 16)
        for (int64_t v = 0; v < n; v++) {
            decode_row(X, v, q);
            int cnt = 0;
            for (int64_t id = 0; id < n; id++) {
                if (id == v) continue;
                decode_row(X, id, x);
                ent e;
                e.d = vdist(q, x, d, X->metric, &e.s);
                e.id = (uint32_t)id;
                e.exp = 0;
                if (cnt == K + 1 && ent_cmp(&e, &best[K]) >= 0) continue;
                int pos = cnt < K + 1 ? cnt++ : K;
                while (pos > 0 && ent_cmp(&e, &best[pos - 1]) < 0) {
                    best[pos] = best[pos - 1];
                    pos--;
                }
                best[pos] = e;
            }
            double g = INFINITY;
            for (int i = 0; i + 1 < cnt; i++) {
                double gi = rel_gap(best[i].d, best[i].s, best[i + 1].d, best[i + 1].s);
                if (gi < g) g = gi;
            }
            kgap[v] = g;
            for (int i = 0; i < K; i++) {
                knn[v * K + i] = best[i].id;
                knd[v * K + i] = best[i].d;
                kns[v * K + i] = best[i].s;
            }
        }
        free(q);
        free(x);
        free(best);
    }
#pragma omp parallel
    {
        double *xa = (double *)malloc(sizeof(double) * d);
        double *xb = (double *)malloc(sizeof(double) * d);
        ent *c = (ent *)malloc(sizeof(ent) * (K > 0 ? K : 1));
#pragma omp for schedule(dynamic, 16)
        for (int64_t v = 0; v < n; v++) {
            for (int i = 0; i < K; i++) {
                c[i].id = knn[v * K + i];
                c[i].d = knd[v * K + i];
                c[i].s = kns[v * K + i];
                c[i].exp = 0;
            }
            double g = prune_core(X, c, K, mode, knn, K, R, graph + v * R, xa, xb);
            if (rows_gap) rows_gap[v] = g < kgap[v] ? g : kgap[v];
        }
        free(xa);
        free(xb);
        free(c);
    }
    free(knn);
    free(knd);
    free(kns);
    free(kgap);
}

/* ------------------------------------------------------------------ */
/* Search (Algorithm 1), one query.  Fills pool[0..*pool_n) sorted by
   (dist, id); returns the smallest decisive relative gap.  n_used bounds
   the ids that exist; graph entries >= n_used are treated as empty. */
typedef struct {
    int64_t n_used;
    const uint32_t *graph;
    int32_t R;
    const uint32_t *del;
    int32_t L, T, k;
    uint64_t seed;
    int32_t W;  /* parents expanded per iteration (0 or 1: Alg. 1 as printed) */
} srch_ctx;

typedef struct {
    int32_t iters;   /* iterations that expanded a parent */
    int64_t evals;   /* distinct distance evaluations */
} srch_stat;

/* Per-iteration features of the learned stop and the trace that trains it.
   After the merge of iteration t (0-based), with the pool sorted, kk =
   min(k, |pool|), d1 / dk / dL the distances at ranks 0 / kk-1 / last,
   s0 = dL - d1 of the initial pool (1 if not positive), the values before
   this iteration's merge marked _prev, and the initial d1 marked _0:
     f0 (t+1)/T            f1 (d1_0 - d1)/s0      f2 (dk - d1)/s0
     f3 (dL - d1)/s0       f4 (mean_k - d1)/s0    f5 std_k/s0
     f6 admitted/R         f7 unexpanded/L        f8 newtop/k
     f9 (t - t_last)/T     f10 expanded/L         f11 parent rank/L
     f12 (dk_prev - dk)/s0 f13 (d1_prev - d1)/s0  f14 (d_next - dk)/s0
     f15 e_t = (e_{t-1} + f6)/2, e_{-1} = 0
   admitted = this iteration's candidates present in the pool after the
   merge; newtop = ids of the new top-kk absent from the previous top-kk;
   t_last = last iteration whose merge changed the top-kk set (-1 before);
   d_next = distance of the nearest unexpanded entry after the merge (the
   next parent), or dL when every entry is expanded.
   mean_k / std_k: mean and population standard deviation of the top-kk.
   The stop network is p = sigmoid(z), z = w2 . relu(W1 f + b1) + b2; it is
   evaluated after iteration t when t+1 >= t_min and (t+1-t_min) is a
   multiple of t_every, and the search stops there if z >= logit(tau). */
#define NFEAT 16
#define NHID 64
typedef struct {
    double *feat;         /* [T][NFEAT] out, or NULL */
    int32_t n_feat;       /* rows written */
    int32_t t_last;       /* last top-k change */
    const double *W1, *b1, *w2; /* stop network (NULL: no stop) */
    double b2, z_tau;
    int32_t t_min;
    int32_t t_every;      /* evaluate the network every t_every iterations (>= 1) */
    double margin;        /* min |z - z_tau| over evaluated iterations */
    int32_t stop_iter;    /* iterations run when stopped, -1 if never */
} feat_ctx;

static double mlp_z(const double *W1, const double *b1, const double *w2, double b2, const double *f) {
    double z = b2;
    for (int j = 0; j < NHID; j++) {
        double h = b1[j];
        for (int i = 0; i < NFEAT; i++) h += W1[j * NFEAT + i] * f[i];
        if (h > 0.0) z += w2[j] * h;
    }
    return z;
}

static double search_one(const orc_store *X, const srch_ctx *S, const double *q, uint64_t qkey, ent *pool,
                         int *pool_n, srch_stat *st, double *x, ent *buf, feat_ctx *F) {
    int d = X->d, L = S->L, R = S->R;
    idset vis;
    set_init(&vis, (int64_t)L + (int64_t)S->T * R);
    double gap = INFINITY;
    int np = 0;
    st->iters = 0;
    st->evals = 0;

    /* InitCandidatePool: L distinct live ids from the draw sequence. */
    uint64_t base = splitmix64(S->seed ^ splitmix64(qkey));
    for (int64_t j = 0; j < 4 * (int64_t)L && np < L && S->n_used > 0; j++) {
        uint32_t id = (uint32_t)(((splitmix64(base ^ (uint64_t)j) >> 32) * (uint64_t)S->n_used) >> 32);
        if (is_deleted(S->del, id) || set_has(&vis, id)) continue;
        set_add(&vis, id);
        decode_row(X, id, x);
        pool[np].d = vdist(q, x, d, X->metric, &pool[np].s);
        pool[np].id = id;
        pool[np].exp = 0;
        np++;
        st->evals++;
    }
    qsort(pool, (size_t)np, sizeof(ent), ent_cmp);

    /* learned-stop bookkeeping */
    double d1_0 = np ? pool[0].d : 0.0, s0 = np ? pool[np - 1].d - pool[0].d : 0.0, ema = 0.0;
    if (!(s0 > 0.0)) s0 = 1.0;
    int t_last = -1;
    if (F) {
        F->n_feat = 0;
        F->margin = INFINITY;
        F->stop_iter = -1;
    }

    const int W = S->W > 1 ? S->W : 1;
    for (int t = 0; t < S->T; t++) {
        /* GetNearest, widened to the W nearest unexpanded entries (W = 1 is
           Alg. 1): par[] lists them in (dist, id) order; pn is the next
           unexpanded entry, which decides the last parent against it. */
        int par[ORC_MAX_W], npar = 0, pn = -1;
        for (int i = 0; i < np; i++)
            if (!pool[i].exp) {
                if (npar < W) par[npar++] = i;
                else { pn = i; break; }
            }
        if (npar == 0) break; /* nothing left to expand: the pool stays unchanged */
        int p = par[0];
        if (pn >= 0) {
            double gi = rel_gap(pool[par[npar - 1]].d, pool[par[npar - 1]].s, pool[pn].d, pool[pn].s);
            if (gi < gap) gap = gi;
        }
        for (int j = 0; j < npar; j++) pool[par[j]].exp = 1;
        st->iters += npar;
        int nb = np;
        memcpy(buf, pool, sizeof(ent) * np);
        /* the parents' rows in turn; an id named by two parents is visited once */
        for (int j = 0; j < npar; j++) {
            const uint32_t *row = S->graph + (int64_t)pool[par[j]].id * R;
            for (int r = 0; r < R; r++) {
                uint32_t v = row[r];
                if (v == ORC_EMPTY || (int64_t)v >= S->n_used) continue;
                if (is_deleted(S->del, v) || set_has(&vis, v)) continue;
                set_add(&vis, v);
                decode_row(X, v, x);
                buf[nb].d = vdist(q, x, d, X->metric, &buf[nb].s);
                buf[nb].id = v;
                buf[nb].exp = 0;
                nb++;
                st->evals++;
            }
        }
        int k = S->k;
        int kk_prev = np < k ? np : k;
        double d1_prev = np ? pool[0].d : 0.0, dk_prev = np ? pool[kk_prev - 1].d : 0.0;
        uint32_t *old_top = F ? (uint32_t *)malloc(sizeof(uint32_t) * (kk_prev > 0 ? kk_prev : 1)) : NULL;
        for (int i = 0; F && i < kk_prev; i++) old_top[i] = pool[i].id;
        int ncand = nb - np;
        for (int i = np; i < nb; i++) buf[i].exp = 2; /* 2 marks "new this iteration" */
        qsort(buf, (size_t)nb, sizeof(ent), ent_cmp);
        if (nb > L) {
            double gi = rel_gap(buf[L - 1].d, buf[L - 1].s, buf[L].d, buf[L].s);
            if (gi < gap) gap = gi;
        }
        np = nb < L ? nb : L;
        memcpy(pool, buf, sizeof(ent) * np);
        int admitted = 0, unexp = 0;
        for (int i = 0; i < np; i++) {
            if (pool[i].exp == 2) { admitted++; pool[i].exp = 0; }
            if (!pool[i].exp) unexp++;
        }
        (void)ncand;
        if (F) {
            int kk = np < k ? np : k, newtop = 0;
            for (int i = 0; i < kk; i++) {
                int found = 0;
                for (int j = 0; j < kk_prev; j++) found |= old_top[j] == pool[i].id;
                newtop += !found;
            }
            free(old_top);
            if (newtop > 0) t_last = t;
            double d1 = pool[0].d, dk = pool[kk - 1].d, dL = pool[np - 1].d, mean = 0.0, var = 0.0;
            for (int i = 0; i < kk; i++) mean += pool[i].d;
            mean /= kk;
            for (int i = 0; i < kk; i++) var += (pool[i].d - mean) * (pool[i].d - mean);
            var /= kk;
            double f[NFEAT];
            f[0] = (double)(t + 1) / S->T;
            f[1] = (d1_0 - d1) / s0;
            f[2] = (dk - d1) / s0;
            f[3] = (dL - d1) / s0;
            f[4] = (mean - d1) / s0;
            f[5] = sqrt(var) / s0;
            f[6] = (double)admitted / R;
            f[7] = (double)unexp / L;
            f[8] = (double)newtop / k;
            f[9] = (double)(t - t_last) / S->T;
            f[10] = (double)(np - unexp) / L;
            f[11] = (double)p / L;
            f[12] = (dk_prev - dk) / s0;
            f[13] = (d1_prev - d1) / s0;
            double d_next = dL;
            for (int i = 0; i < np; i++)
                if (!pool[i].exp) {
                    d_next = pool[i].d;
                    break;
                }
            f[14] = (d_next - dk) / s0;
            ema = 0.5 * ema + 0.5 * f[6];
            f[15] = ema;
            if (F->feat) memcpy(F->feat + (int64_t)t * NFEAT, f, sizeof(f));
            F->n_feat = t + 1;
            F->t_last = t_last;
            if (F->W1 && t + 1 >= F->t_min && (t + 1 - F->t_min) % (F->t_every > 0 ? F->t_every : 1) == 0) {
                double z = mlp_z(F->W1, F->b1, F->w2, F->b2, f);
                double mg = fabs(z - F->z_tau);
                if (mg < F->margin) F->margin = mg;
                if (z >= F->z_tau) {
                    F->stop_iter = t + 1;
                    break;
                }
            }
        }
    }
    /* output order and the k-boundary */
    for (int i = 0; i + 1 < np && i < S->k; i++) {
        double gi = rel_gap(pool[i].d, pool[i].s, pool[i + 1].d, pool[i + 1].s);
        if (gi < gap) gap = gi;
    }
    set_free(&vis);
    *pool_n = np;
    return gap;
}

/* Batched search, W parents per iteration (1 <= W <= ORC_MAX_W; W = 1 is
   Alg. 1).  Outputs (each optional except ids):
     out_ids/out_d [nq][k]  (EMPTY / +inf pad), out_gap[nq], out_iters[nq]
     (parents expanded), out_evals[nq], pool_ids/pool_d [nq][L] (the final
     pool, EMPTY / +inf pad).  Returns -1 for W out of range. */
int orc_search(const orc_store *X, int64_t n_used, const uint32_t *graph, int32_t R, const uint32_t *del,
               const void *Q, int64_t nq, const uint64_t *qkeys, int32_t k, int32_t L, int32_t T, uint64_t seed,
               int32_t W, uint32_t *out_ids, double *out_d, double *out_gap, int32_t *out_iters, int64_t *out_evals,
               uint32_t *pool_ids, double *pool_d) {
    if (W < 1 || W > ORC_MAX_W) return -1;
    srch_ctx S = {n_used, graph, R, del, L, T, k, seed, W};
    int d = X->d;
    int64_t qb = query_bytes(X);
#pragma omp parallel
    {
        double *q = (double *)malloc(sizeof(double) * d);
        double *x = (double *)malloc(sizeof(double) * d);
        ent *pool = (ent *)malloc(sizeof(ent) * (L + (size_t)W * R + 1));
        ent *buf = (ent *)malloc(sizeof(ent) * (L + (size_t)W * R + 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t qi = 0; qi < nq; qi++) {
            decode_query(X, Q, qi, q);
            uint64_t key = qkeys ? qkeys[qi] : orc_query_key((const uint8_t *)Q + qi * qb, qb);
            int np;
            srch_stat st;
            double g = search_one(X, &S, q, key, pool, &np, &st, x, buf, NULL);
            for (int i = 0; i < k; i++) {
                out_ids[qi * k + i] = i < np ? pool[i].id : ORC_EMPTY;
                if (out_d) out_d[qi * k + i] = i < np ? pool[i].d : INFINITY;
            }
            if (out_gap) out_gap[qi] = g;
            if (out_iters) out_iters[qi] = st.iters;
            if (out_evals) out_evals[qi] = st.evals;
            if (pool_ids)
                for (int i = 0; i < L; i++) {
                    pool_ids[qi * L + i] = i < np ? pool[i].id : ORC_EMPTY;
                    if (pool_d) pool_d[qi * L + i] = i < np ? pool[i].d : INFINITY;
                }
        }
        free(q);
        free(x);
        free(pool);
        free(buf);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Insert (Sec. 5.1), one batch of m vectors already written to store rows
   [n0, n0+m).  Every new vertex searches the pre-batch graph (n0 vertices,
   pool size L_ins, T_ins iterations, key = its query key); its live pool is
   reordered (orc_prune, N_out = pre-batch rows) into its row.  Then each
   old vertex u named by new rows gets its tail half [R/2, R) replaced by the
   R/2 best, by (dist, id), of its live tail entries and the new vertices
   that chose it; remaining tail slots become EMPTY; the head half is kept.
   Rows are written after all of them are computed.
   new_gap[m]: smallest decisive gap of each new row (search + prune);
   tail_gap[n0]: for patched old rows, the smallest gap of the tail merge
   (INFINITY where untouched).  Optional. */
typedef struct {
    uint32_t target, src;
    double d, s;
} revreq;

static int rev_cmp(const void *pa, const void *pb) {
    const revreq *a = (const revreq *)pa, *b = (const revreq *)pb;
    if (a->target != b->target) return (a->target > b->target) - (a->target < b->target);
    if (a->d < b->d) return -1;
    if (a->d > b->d) return 1;
    return (a->src > b->src) - (a->src < b->src);
}

/* Reverse edges of new vertices n0 .. n0+m-1 whose rows are rows[m][R], with
   rowd / rows_s the distances (and scales) of those entries: every named
   target u < tmax keeps as its tail half [R/2, R) the R/2 best (dist, id) of
   its live tail entries (ids < n0) and the new vertices that chose it; the
   head half is kept.  tail_gap (optional): per target, the smallest decisive
   gap of its merge (INFINITY for untouched u < tmax). */
static void reverse_patch(const orc_store *X, uint32_t *graph, int32_t R, const uint32_t *del, int64_t n0,
                          int64_t m, const uint32_t *rows, const double *rowd, const double *rows_s, int64_t tmax,
                          double *tail_gap) {
    int d = X->d;
    /* reverse-edge requests (u, v, dist(u, v)) */
    int64_t nreq = 0;
    revreq *req = (revreq *)malloc(sizeof(revreq) * (size_t)(m > 0 ? m : 1) * R);
    for (int64_t i = 0; i < m; i++)
        for (int r = 0; r < R; r++) {
            uint32_t u = rows[i * R + r];
            if (u == ORC_EMPTY || (int64_t)u >= tmax) continue;
            req[nreq].target = u;
            req[nreq].src = (uint32_t)(n0 + i);
            req[nreq].d = rowd[i * R + r];
            req[nreq].s = rows_s[i * R + r];
            nreq++;
        }
    qsort(req, (size_t)nreq, sizeof(revreq), rev_cmp);
    if (tail_gap)
        for (int64_t u = 0; u < tmax; u++) tail_gap[u] = INFINITY;
    int H = R / 2, TL = R - R / 2;
    /* group starts */
    int64_t ngrp = 0;
    int64_t *gs = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nreq + 1));
    for (int64_t a = 0; a < nreq; a++)
        if (a == 0 || req[a].target != req[a - 1].target) gs[ngrp++] = a;
    gs[ngrp] = nreq;
#pragma omp parallel
    {
        double *xa = (double *)malloc(sizeof(double) * d);
        double *xb = (double *)malloc(sizeof(double) * d);
        ent *mg = (ent *)malloc(sizeof(ent) * (size_t)(TL + m + 1));
#pragma omp for schedule(dynamic, 16)
        for (int64_t g = 0; g < ngrp; g++) {
            uint32_t u = req[gs[g]].target;
            uint32_t *row = graph + (int64_t)u * R;
            int nm = 0;
            decode_row(X, u, xa);
            for (int r = H; r < R; r++) {
                uint32_t t = row[r];
                if (t == ORC_EMPTY || (int64_t)t >= n0 || is_deleted(del, t)) continue;
                decode_row(X, t, xb);
                mg[nm].d = vdist(xa, xb, d, X->metric, &mg[nm].s);
                mg[nm].id = t;
                mg[nm].exp = 0;
                nm++;
            }
            for (int64_t a = gs[g]; a < gs[g + 1]; a++) {
                mg[nm].d = req[a].d;
                mg[nm].s = req[a].s;
                mg[nm].id = req[a].src;
                mg[nm].exp = 0;
                nm++;
            }
            qsort(mg, (size_t)nm, sizeof(ent), ent_cmp);
            double gp = INFINITY;
            for (int i = 0; i + 1 < nm && i < TL; i++) {
                double gi = rel_gap(mg[i].d, mg[i].s, mg[i + 1].d, mg[i + 1].s);
                if (gi < gp) gp = gi;
            }
            if (tail_gap) tail_gap[u] = gp;
            for (int r = 0; r < TL; r++) row[H + r] = r < nm ? mg[r].id : ORC_EMPTY;
        }
        free(xa);
        free(xb);
        free(mg);
    }
    free(gs);
    free(req);
}

void orc_insert(const orc_store *X, int64_t n0, int64_t m, uint32_t *graph, int32_t R, const uint32_t *del,
                int32_t L_ins, int32_t T_ins, uint64_t seed, int32_t mode, double *new_gap, double *tail_gap) {
    int d = X->d;
    srch_ctx S = {n0, graph, R, del, L_ins, T_ins, L_ins, seed};
    uint32_t *rows = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1) * R);
    double *rowd = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1) * R);
    double *rows_s = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1) * R);
#pragma omp parallel
    {
        double *q = (double *)malloc(sizeof(double) * d);
        double *x = (double *)malloc(sizeof(double) * d);
        double *xb = (double *)malloc(sizeof(double) * d);
        ent *pool = (ent *)malloc(sizeof(ent) * (L_ins + R + 1));
        ent *buf = (ent *)malloc(sizeof(ent) * (L_ins + R + 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < m; i++) {
            int64_t v = n0 + i;
            const uint8_t *raw = (const uint8_t *)X->data + v * X->pitch;
            uint64_t key = orc_query_key(raw, query_bytes(X));
            decode_row(X, v, q);
            int np;
            srch_stat st;
            double g = search_one(X, &S, q, key, pool, &np, &st, x, buf, NULL);
            uint32_t *out = rows + i * R;
            double g2 = prune_core(X, pool, np, mode, graph, R, R, out, x, xb);
            if (g2 < g) g = g2;
            for (int r = 0; r < R; r++) {
                rowd[i * R + r] = INFINITY;
                rows_s[i * R + r] = 0.0;
                for (int j = 0; j < np; j++)
                    if (pool[j].id == out[r]) {
                        rowd[i * R + r] = pool[j].d;
                        rows_s[i * R + r] = pool[j].s;
                        break;
                    }
            }
            if (new_gap) new_gap[i] = g;
        }
        free(q);
        free(x);
        free(xb);
        free(pool);
        free(buf);
    }
    reverse_patch(X, graph, R, del, n0, m, rows, rowd, rows_s, n0, tail_gap);
    for (int64_t i = 0; i < m; i++) memcpy(graph + (n0 + i) * R, rows + i * R, sizeof(uint32_t) * R);
    free(rows);
    free(rowd);
    free(rows_s);
}

/* Repair (Sec. 5.2) of every live vertex u < n_used whose snapshot row has
   at least min_del deleted entries: candidates = u's live row entries in row
   order, then for each deleted p in u's row (row order) the first c entries
   of N_out(p) that are live, not u and not yet candidates, at most cap in
   all; sorted by (dist(u, .), id); reordered by prune_core (N_out from the
   snapshot); if fewer than R survive, u's deleted entries fill the remaining
   slots in their original order (then EMPTY).  Reads only snap, writes the
   new rows into graph.  With `only`, just the rows only[0 .. n_only) are
   considered and row i of graph / rows_gap stands for vertex only[i].
   Returns the number of rewritten rows. */
static int64_t repair_rows(const orc_store *X, int64_t n_used, uint32_t *graph, const uint32_t *snap, int32_t R,
                           const uint32_t *del, int32_t c, int32_t min_del, int32_t cap, int32_t mode,
                           double *rows_gap, const uint32_t *only, int64_t n_only) {
    int d = X->d;
    int64_t nrep = 0;
    const int64_t count = only ? n_only : n_used;
    if (rows_gap)
        for (int64_t i = 0; i < count; i++) rows_gap[i] = INFINITY;
#pragma omp parallel reduction(+ : nrep)
    {
        double *xa = (double *)malloc(sizeof(double) * d);
        double *xb = (double *)malloc(sizeof(double) * d);
        ent *cd = (ent *)malloc(sizeof(ent) * cap);
        uint32_t *out = (uint32_t *)malloc(sizeof(uint32_t) * R);
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < count; i++) {
            const int64_t u = only ? (int64_t)only[i] : i;
            if (is_deleted(del, (uint32_t)u)) continue;
            const uint32_t *row = snap + u * R;
            int nd = 0;
            for (int r = 0; r < R; r++)
                if (row[r] != ORC_EMPTY && is_deleted(del, row[r])) nd++;
            if (nd < min_del) continue;
            int nc = 0;
            for (int r = 0; r < R; r++) {
                uint32_t t = row[r];
                if (t == ORC_EMPTY || is_deleted(del, t) || t == (uint32_t)u) continue;
                int dup = 0;
                for (int j = 0; j < nc; j++) dup |= cd[j].id == t;
                if (!dup) cd[nc++].id = t;
            }
            for (int r = 0; r < R; r++) {
                uint32_t p = row[r];
                if (p == ORC_EMPTY || !is_deleted(del, p)) continue;
                const uint32_t *prow = snap + (int64_t)p * R;
                int taken = 0;
                for (int s = 0; s < R && taken < c && nc < cap; s++) {
                    uint32_t w = prow[s];
                    if (w == ORC_EMPTY || is_deleted(del, w) || w == (uint32_t)u) continue;
                    int dup = 0;
                    for (int j = 0; j < nc; j++) dup |= cd[j].id == w;
                    if (dup) continue;
                    cd[nc++].id = w;
                    taken++;
                }
            }
            decode_row(X, u, xa);
            for (int j = 0; j < nc; j++) {
                decode_row(X, cd[j].id, xb);
                cd[j].d = vdist(xa, xb, d, X->metric, &cd[j].s);
                cd[j].exp = 0;
            }
            qsort(cd, (size_t)nc, sizeof(ent), ent_cmp);
            double g = INFINITY;
            for (int j = 0; j + 1 < nc; j++) {
                double gi = rel_gap(cd[j].d, cd[j].s, cd[j + 1].d, cd[j + 1].s);
                if (gi < g) g = gi;
            }
            double g2 = prune_core(X, cd, nc, mode, snap, R, R, out, xa, xb);
            if (g2 < g) g = g2;
            int w = nc < R ? nc : R;
            for (int r = 0; r < R && w < R; r++)
                if (row[r] != ORC_EMPTY && is_deleted(del, row[r])) out[w++] = row[r];
            uint32_t *dst = graph + i * R;
            memcpy(dst, out, sizeof(uint32_t) * R);
            if (rows_gap) rows_gap[i] = g;
            nrep++;
        }
        free(xa);
        free(xb);
        free(cd);
        free(out);
    }
    return nrep;
}


/* ------------------------------------------------------------------ */
/* Delete (Sec. 5.2).  Returns the number of newly deleted ids, or -1 when
   some id >= n_used (nothing is changed then).  After marking, every live
   vertex u with more than half (strictly, 2*#deleted > R) of its row deleted
   is repaired from a snapshot of the graph:
     candidates = u's live row entries in row order, then for each deleted
     p in u's row (row order) the first c entries of N_out(p) that are live,
     not u and not yet candidates; sorted by (dist(u, .), id); reordered by
     orc_prune; if fewer than R survive, u's deleted entries fill the
     remaining slots in their original order (then EMPTY).
   out_repaired (optional): number of repaired rows.  rows_gap[n_used]
   (optional): smallest decisive gap of each repaired row (INFINITY
   elsewhere). */
int64_t orc_delete(const orc_store *X, int64_t n_used, uint32_t *graph, int32_t R, uint32_t *del,
                   const uint32_t *ids, int64_t m, int32_t c, int32_t mode, int64_t *out_repaired,
                   double *rows_gap) {
    for (int64_t i = 0; i < m; i++)
        if ((int64_t)ids[i] >= n_used) return -1;
    int64_t newly = 0;
    for (int64_t i = 0; i < m; i++)
        if (!is_deleted(del, ids[i])) {
            del[ids[i] >> 5] |= 1u << (ids[i] & 31);
            newly++;
        }
    uint32_t *snap = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n_used > 0 ? n_used : 1) * R);
    memcpy(snap, graph, sizeof(uint32_t) * (size_t)n_used * R);
    int64_t nrep = repair_rows(X, n_used, graph, snap, R, del, c, R / 2 + 1, R + c * R, mode, rows_gap, NULL, 0);
    free(snap);
    if (out_repaired) *out_repaired = nrep;
    return newly;
}

/* Global consolidation (Sec. 5.2), on the snapshot of Sec. 5.3's
   multi-version mechanism: graph holds rows [0, n0) and del the deletion
   bits of the moment the snapshot was taken.  Every live vertex with at
   least one deleted out-neighbour is repaired as in orc_delete, taking every
   live entry of each deleted neighbour's row (c = R), at most cap candidates
   in all (u's live entries first, then the deleted neighbours in row order,
   each row in order; cap >= R).  Returns the number of rewritten rows, or -1
   for cap < R. */
int64_t orc_consolidate(const orc_store *X, int64_t n0, uint32_t *graph, int32_t R, const uint32_t *del, int32_t cap,
                        int32_t mode, double *rows_gap) {
    if (cap < R) return -1; /* u's own live entries always fit */
    uint32_t *snap = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n0 > 0 ? n0 : 1) * R);
    memcpy(snap, graph, sizeof(uint32_t) * (size_t)n0 * R);
    int64_t nrep = repair_rows(X, n0, graph, snap, R, del, R, 1, cap, mode, rows_gap, NULL, 0);
    free(snap);
    return nrep;
}

/* orc_consolidate for the rows only[0 .. n_only) alone, from the unchanged
   graph (read only): out_rows[i] = the consolidated row of vertex only[i]
   (its current row when it is deleted or names no deleted vertex); rows_gap
   per listed row.  For sampled checks of a large graph.  -1 for cap < R. */
int64_t orc_consolidate_rows(const orc_store *X, int64_t n0, const uint32_t *graph, int32_t R, const uint32_t *del,
                             int32_t cap, int32_t mode, const uint32_t *only, int64_t n_only, uint32_t *out_rows,
                             double *rows_gap) {
    if (cap < R) return -1;
    for (int64_t i = 0; i < n_only; i++) memcpy(out_rows + i * R, graph + (int64_t)only[i] * R, sizeof(uint32_t) * R);
    return repair_rows(X, n0, out_rows, graph, R, del, R, 1, cap, mode, rows_gap, only, n_only);
}

/* Reverse Edge Integration (Sec. 5.3): the logged reverse edges of one insert
   batch (new vertices n0 .. n0+m-1 with graph rows rows[m][R]) applied to a
   consolidated graph; distances are recomputed here; targets >= tmax (rows
   that are not part of the consolidated snapshot) are skipped. */
void orc_reverse_patch(const orc_store *X, uint32_t *graph, int32_t R, const uint32_t *del, int64_t n0, int64_t m,
                       const uint32_t *rows, int64_t tmax, double *tail_gap) {
    int d = X->d;
    double *rowd = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1) * R);
    double *rows_s = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1) * R);
#pragma omp parallel
    {
        double *xa = (double *)malloc(sizeof(double) * d);
        double *xb = (double *)malloc(sizeof(double) * d);
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < m; i++) {
            decode_row(X, n0 + i, xa);
            for (int r = 0; r < R; r++) {
                uint32_t u = rows[i * R + r];
                rowd[i * R + r] = INFINITY;
                rows_s[i * R + r] = 0.0;
                if (u == ORC_EMPTY) continue;
                decode_row(X, u, xb);
                rowd[i * R + r] = vdist(xa, xb, d, X->metric, &rows_s[i * R + r]);
            }
        }
        free(xa);
        free(xb);
    }
    reverse_patch(X, graph, R, del, n0, m, rows, rowd, rows_s, tmax, tail_gap);
    free(rowd);
    free(rows_s);
}

/* ------------------------------------------------------------------ */
int32_t orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int32_t t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ------------------------------------------------------------------ */
/* Search with the learned stop and/or the per-iteration trace.
   feat [nq][T][16] (optional) receives the features of every iteration run;
   n_feat[nq] the number of rows written; t_last[nq] the last iteration that
   changed the top-k set (labels: y_t = t >= t_last).  When W1 != NULL the
   stop network (weights as given, FP64 arithmetic) ends a query after
   iteration t once t+1 >= t_min, (t+1-t_min) % t_every == 0 and z >= z_tau;
   stop_iter[nq] = iterations
   run (-1: never stopped), margin[nq] = min |z - z_tau| seen. */
void orc_search_ex(const orc_store *X, int64_t n_used, const uint32_t *graph, int32_t R, const uint32_t *del,
                   const void *Q, int64_t nq, const uint64_t *qkeys, int32_t k, int32_t L, int32_t T, uint64_t seed,
                   uint32_t *out_ids, double *out_d, double *out_gap, double *feat, int32_t *n_feat,
                   int32_t *t_last, const double *W1, const double *b1, const double *w2, double b2, double z_tau,
                   int32_t t_min, int32_t t_every, int32_t *stop_iter, double *margin) {
    srch_ctx S = {n_used, graph, R, del, L, T, k, seed};
    int d = X->d;
    int64_t qb = query_bytes(X);
#pragma omp parallel
    {
        double *q = (double *)malloc(sizeof(double) * d);
        double *x = (double *)malloc(sizeof(double) * d);
        ent *pool = (ent *)malloc(sizeof(ent) * (L + R + 1));
        ent *buf = (ent *)malloc(sizeof(ent) * (L + R + 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t qi = 0; qi < nq; qi++) {
            decode_query(X, Q, qi, q);
            uint64_t key = qkeys ? qkeys[qi] : orc_query_key((const uint8_t *)Q + qi * qb, qb);
            int np;
            srch_stat st;
            feat_ctx F;
            memset(&F, 0, sizeof(F));
            F.feat = feat ? feat + qi * (int64_t)T * NFEAT : NULL;
            F.W1 = W1;
            F.b1 = b1;
            F.w2 = w2;
            F.b2 = b2;
            F.z_tau = z_tau;
            F.t_min = t_min;
            F.t_every = t_every;
            double g = search_one(X, &S, q, key, pool, &np, &st, x, buf, &F);
            for (int i = 0; i < k; i++) {
                out_ids[qi * k + i] = i < np ? pool[i].id : ORC_EMPTY;
                if (out_d) out_d[qi * k + i] = i < np ? pool[i].d : INFINITY;
            }
            if (out_gap) out_gap[qi] = g;
            if (n_feat) n_feat[qi] = F.n_feat;
            if (t_last) t_last[qi] = F.t_last;
            if (stop_iter) stop_iter[qi] = F.stop_iter;
            if (margin) margin[qi] = F.margin;
        }
        free(q);
        free(x);
        free(pool);
        free(buf);
    }
}

/* Distances from each query to given ids (EMPTY -> +inf): out[nq][k]. */
void orc_dist_ids(const orc_store *X, const void *Q, int64_t nq, const uint32_t *ids, int32_t k, double *out) {
    int d = X->d;
#pragma omp parallel
    {
        double *q = (double *)malloc(sizeof(double) * d);
        double *x = (double *)malloc(sizeof(double) * d);
#pragma omp for schedule(static)
        for (int64_t qi = 0; qi < nq; qi++) {
            decode_query(X, Q, qi, q);
            for (int i = 0; i < k; i++) {
                uint32_t id = ids[qi * k + i];
                if (id == ORC_EMPTY || (int64_t)id >= X->n) {
                    out[qi * k + i] = INFINITY;
                    continue;
                }
                double s;
                decode_row(X, id, x);
                out[qi * k + i] = vdist(q, x, d, X->metric, &s);
            }
        }
        free(q);
        free(x);
    }
}

/* Stop network forward: z[nb] and p[nb] = sigmoid(z). */
void orc_mlp_forward(const double *W1, const double *b1, const double *w2, double b2, const double *F, int64_t nb,
                     double *z, double *p) {
    for (int64_t s = 0; s < nb; s++) {
        double zs = mlp_z(W1, b1, w2, b2, F + s * NFEAT);
        if (z) z[s] = zs;
        if (p) p[s] = 1.0 / (1.0 + exp(-zs));
    }
}

/* Mean binary cross-entropy over the batch and its gradients:
   loss = mean_s [ softplus(z_s) - y_s z_s ],  dL/dz_s = (sigmoid(z_s) - y_s)/nb,
   back through z = w2 . relu(h) + b2, h = W1 f + b1.  Gradients are
   overwritten.  Returns the loss. */
double orc_mlp_backward(const double *W1, const double *b1, const double *w2, double b2, const double *F,
                        const double *y, int64_t nb, double *gW1, double *gb1, double *gw2, double *gb2) {
    memset(gW1, 0, sizeof(double) * NHID * NFEAT);
    memset(gb1, 0, sizeof(double) * NHID);
    memset(gw2, 0, sizeof(double) * NHID);
    *gb2 = 0.0;
    double loss = 0.0, h[NHID];
    for (int64_t s = 0; s < nb; s++) {
        const double *f = F + s * NFEAT;
        double z = b2;
        for (int j = 0; j < NHID; j++) {
            h[j] = b1[j];
            for (int i = 0; i < NFEAT; i++) h[j] += W1[j * NFEAT + i] * f[i];
            if (h[j] > 0.0) z += w2[j] * h[j];
        }
        double sp = z > 0 ? z + log1p(exp(-z)) : log1p(exp(z));
        loss += sp - y[s] * z;
        double dz = (1.0 / (1.0 + exp(-z)) - y[s]) / (double)nb;
        *gb2 += dz;
        for (int j = 0; j < NHID; j++) {
            if (h[j] <= 0.0) continue;
            gw2[j] += dz * h[j];
            double dh = dz * w2[j];
            gb1[j] += dh;
            for (int i = 0; i < NFEAT; i++) gW1[j * NFEAT + i] += dh * f[i];
        }
    }
    return loss / (double)nb;
}

/* ------------------------------------------------------------------ */
/* One maintenance round of workload-aware vector placement (Sec. 4.3,
   Eq. 2, Alg. 2), batched: F(x) = alpha*freq(x) + beta*log(1 + ein(x)).
   Candidates: queue[0..c) ordered by descending F (ties: ascending id), the
   first B.  Victims: the W slots from the clock hand (mod M); a referenced
   slot loses its bit and is passed over (second chance); the unreferenced
   ones are ordered by ascending F of their owner (an empty slot first,
   ties: ascending slot); if fewer than B were unreferenced the clock comes
   round the window again, when every slot in it is unreferenced (Alg. 2's
   sweep continues until it finds a victim).  The i-th candidate replaces the i-th victim for
   i < min(B, #victims): the evicted owner's map entry becomes -1, the
   candidate maps to the slot, and the slot's reference bit is set. */
typedef struct {
    double f;
    int64_t k;
} fk;
static int fk_desc(const void *pa, const void *pb) {
    const fk *a = (const fk *)pa, *b = (const fk *)pb;
    if (a->f != b->f) return a->f > b->f ? -1 : 1;
    return (a->k > b->k) - (a->k < b->k);
}
static int fk_asc(const void *pa, const void *pb) {
    const fk *a = (const fk *)pa, *b = (const fk *)pb;
    if (a->f != b->f) return a->f < b->f ? -1 : 1;
    return (a->k > b->k) - (a->k < b->k);
}
void orc_wavp_round(int64_t M, int32_t *map, int32_t *owner, uint8_t *ref, const uint32_t *freq, const uint32_t *ein,
                    const uint32_t *queue, int64_t c, int64_t B, int64_t hand, int64_t W, double alpha, double beta,
                    int64_t *promoted, int64_t *evicted) {
    fk *cand = (fk *)malloc(sizeof(fk) * (size_t)(c > 0 ? c : 1));
    fk *vic = (fk *)malloc(sizeof(fk) * (size_t)(W > 0 ? W : 1));
    for (int64_t i = 0; i < c; i++) {
        uint32_t x = queue[i];
        cand[i].f = alpha * freq[x] + beta * log(1.0 + ein[x]);
        cand[i].k = x;
    }
    qsort(cand, (size_t)c, sizeof(fk), fk_desc);
    int64_t nv = 0;
    int64_t want = B < c ? B : c;
    for (int pass = 0; pass < 2 && (pass == 0 || nv < want); pass++) {
        nv = 0;
        for (int64_t i = 0; i < W; i++) {
            int64_t s = (hand + i) % M;
            if (ref[s]) {
                ref[s] = 0;
                continue;
            }
            int32_t o = owner[s];
            vic[nv].f = o < 0 ? -INFINITY : alpha * freq[o] + beta * log(1.0 + ein[o]);
            vic[nv].k = s;
            nv++;
        }
    }
    qsort(vic, (size_t)nv, sizeof(fk), fk_asc);
    int64_t np = B < c ? B : c;
    if (nv < np) np = nv;
    *promoted = 0;
    *evicted = 0;
    for (int64_t i = 0; i < np; i++) {
        int64_t s = vic[i].k;
        uint32_t x = (uint32_t)cand[i].k;
        if (owner[s] >= 0) {
            map[owner[s]] = -1;
            (*evicted)++;
        }
        owner[s] = (int32_t)x;
        map[x] = (int32_t)s;
        ref[s] = 1;
        (*promoted)++;
    }
    free(cand);
    free(vic);
}
