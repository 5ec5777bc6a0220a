/*
 * Plain C oracle for OPH / GOPH / (a:b)HOPH / MinWise.
 *
 * TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the
 * CPU-baseline legs of bench.py load this library.  It shares no code,
 * header, table or constant generator with the CUDA library; it is the
 * scalable twin of oracle/hoph_ref.py (exact Fractions), checked against it
 * by the tests.
 *
 * Paper: Zhang et al., "Hierarchical One Permutation Hashing: Efficient
 * Multimedia Near Duplicate Detection" (arXiv 1805.11254).  Section,
 * equation and algorithm numbers below are the paper's; the readings taken
 * where the paper is garbled are the ones listed in oracle/hoph_ref.py.
 *
 * Everything is plain loops over the definitions.  Decisions are taken on
 * exact integer fractions (__int128 cross-multiplication) and the binomial
 * tails are looked up at ceil(m), as Algorithm 1/2 read F(m); whether a tail
 * is <= eps is decided exactly, on the integers td^k' P(X = i) (fixed-size
 * multi-word arithmetic below).  Work is split across POSIX threads by
 * query (comparison) or by set (sketching) only.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_EMPTY 0xFFFFFFFFu
#define OR_P61 ((((uint64_t)1) << 61) - 1)

typedef __int128 i128;

/* ----------------------------------------------------------------------- */
/* SplitMix64 (Steele, Lea, Flood 2014)                                     */
/* ----------------------------------------------------------------------- */

static uint64_t sm64(uint64_t *state) {
    uint64_t z;
    *state += 0x9E3779B97F4A7C15ull;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* psi as an explicit table (Sec. 3.2): Fisher-Yates from the identity,
 * i = D-1 .. 1, j = next() mod (i+1). */
int or_permutation(uint64_t D, uint64_t seed, uint32_t *out) {
    uint64_t s = seed, i;
    if (D == 0 || D > (((uint64_t)1) << 32)) return -1;
    for (i = 0; i < D; ++i) out[i] = (uint32_t)i;
    for (i = D - 1; i >= 1; --i) {
        uint64_t j = sm64(&s) % (i + 1);
        uint32_t t = out[i];
        out[i] = out[j];
        out[j] = t;
    }
    return 0;
}

/* Parameters of the 2-universal hash psi(x) = ((a x + b) mod p) >> 29. */
void or_hash_params(uint64_t seed, uint64_t *a, uint64_t *b) {
    uint64_t s = seed;
    *a = 1 + sm64(&s) % (OR_P61 - 1);
    *b = sm64(&s) % OR_P61;
}

static uint32_t hash_psi(uint64_t x, uint64_t a, uint64_t b) {
    unsigned __int128 v = (unsigned __int128)a * x + b;
    return (uint32_t)((uint64_t)(v % OR_P61) >> 29);
}

uint32_t or_hash_psi(uint64_t x, uint64_t a, uint64_t b) { return hash_psi(x, a, b); }

/* ----------------------------------------------------------------------- */
/* Layout: bin lower bounds lo[0..k], lo[k] = D                             */
/* ----------------------------------------------------------------------- */

static uint64_t ceil_div_u(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

/* a = b = 0: k equal bins over V (Sec. 3.2).  Otherwise (a:b)HOPH
 * (Sec. 4.1): G-1 splits giving floor(rem*a/(a+b)) to the permutation group,
 * the last group takes the remainder; each group split evenly into kg bins. */
int or_layout(uint64_t D, uint32_t k, uint32_t kg, uint32_t a, uint32_t b,
              uint64_t *lo) {
    uint32_t G, g, i;
    if (kg == 0 || k % kg) return -1;
    G = k / kg;
    if (a == 0 && b == 0) {
        uint32_t j;
        if (D < k) return -1;
        for (j = 0; j <= k; ++j)
            lo[j] = (uint64_t)(((unsigned __int128)j * D + k - 1) / k);
        return 0;
    } else {
        uint64_t rem = D, start = 0;
        for (g = 0; g < G; ++g) {
            uint64_t zg = (g + 1 < G)
                ? (uint64_t)(((unsigned __int128)rem * a) / (a + b)) : rem;
            if (zg < kg) return -1;
            for (i = 0; i < kg; ++i)
                lo[g * kg + i] = start + ceil_div_u((uint64_t)i * zg, kg);
            start += zg;
            rem -= zg;
        }
        lo[k] = D;
        return 0;
    }
}

/* index j with lo[j] <= p < lo[j+1] (binary search over the bounds) */
static uint32_t find_bin(const uint64_t *lo, uint32_t k, uint64_t p) {
    uint32_t l = 0, h = k; /* invariant lo[l] <= p < lo[h] */
    while (h - l > 1) {
        uint32_t m = (l + h) / 2;
        if (lo[m] <= p) l = m; else h = m;
    }
    return l;
}

/* ----------------------------------------------------------------------- */
/* Thread helper                                                            */
/* ----------------------------------------------------------------------- */

typedef struct {
    void (*fn)(void *ctx, int64_t begin, int64_t end, int tid);
    void *ctx;
    int64_t begin, end;
    int tid;
} or_job;

static void *or_job_run(void *p) {
    or_job *j = (or_job *)p;
    j->fn(j->ctx, j->begin, j->end, j->tid);
    return 0;
}

static void run_parallel(void (*fn)(void *, int64_t, int64_t, int), void *ctx,
                         int64_t n, int threads) {
    pthread_t th[256];
    or_job jobs[256];
    int t;
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if (n < threads) threads = n > 0 ? (int)n : 1;
    for (t = 0; t < threads; ++t) {
        jobs[t].fn = fn;
        jobs[t].ctx = ctx;
        jobs[t].begin = n * t / threads;
        jobs[t].end = n * (t + 1) / threads;
        jobs[t].tid = t;
    }
    for (t = 1; t < threads; ++t) pthread_create(&th[t], 0, or_job_run, &jobs[t]);
    or_job_run(&jobs[0]);
    for (t = 1; t < threads; ++t) pthread_join(th[t], 0);
}

/* ----------------------------------------------------------------------- */
/* Sketches                                                                 */
/* ----------------------------------------------------------------------- */

typedef struct {
    const uint32_t *ids;
    const int64_t *off;
    const uint32_t *perm; /* NULL: hash */
    uint64_t D, ha, hb;
    const uint64_t *lo;
    uint32_t k;
    uint32_t *out;
    volatile int err;
} sketch_ctx;

static void sketch_range(void *p, int64_t b, int64_t e, int tid) {
    sketch_ctx *c = (sketch_ctx *)p;
    int64_t i, t;
    uint32_t j;
    (void)tid;
    for (i = b; i < e; ++i) {
        uint32_t *sk = c->out + (size_t)i * c->k;
        for (j = 0; j < c->k; ++j) sk[j] = OR_EMPTY;
        for (t = c->off[i]; t < c->off[i + 1]; ++t) {
            uint64_t x = c->ids[t], pv;
            uint32_t bin;
            uint64_t v;
            if (x >= c->D) { c->err = 1; continue; }
            pv = c->perm ? c->perm[x] : hash_psi(x, c->ha, c->hb);
            bin = find_bin(c->lo, c->k, pv);
            v = pv - c->lo[bin];
            if (v < sk[bin]) sk[bin] = (uint32_t)v;
        }
    }
}

/* OPH / HOPH sketches (Sec. 3.2, 4.1) of n sets into out[n][k] (bins in
 * psi-space order).  Returns 0, or -2 if some ID was >= D. */
int or_sketch(const uint32_t *ids, const int64_t *offsets, int64_t n,
              const uint32_t *perm, uint64_t D, uint64_t ha, uint64_t hb,
              const uint64_t *lo, uint32_t k, uint32_t *out, int threads) {
    sketch_ctx c;
    c.ids = ids; c.off = offsets; c.perm = perm; c.D = D; c.ha = ha; c.hb = hb;
    c.lo = lo; c.k = k; c.out = out; c.err = 0;
    run_parallel(sketch_range, &c, n, threads);
    return c.err ? -2 : 0;
}

typedef struct {
    const uint32_t *ids;
    const int64_t *off;
    const uint32_t *perms; /* [k][D] */
    uint64_t D;
    uint32_t k;
    uint32_t *out;
    volatile int err;
} minwise_ctx;

static void minwise_range(void *p, int64_t b, int64_t e, int tid) {
    minwise_ctx *c = (minwise_ctx *)p;
    int64_t i, t;
    uint32_t j;
    (void)tid;
    for (i = b; i < e; ++i) {
        uint32_t *sk = c->out + (size_t)i * c->k;
        for (j = 0; j < c->k; ++j) {
            uint32_t m = OR_EMPTY;
            const uint32_t *psi = c->perms + (size_t)j * c->D;
            for (t = c->off[i]; t < c->off[i + 1]; ++t) {
                uint32_t x = c->ids[t];
                if (x >= c->D) { c->err = 1; continue; }
                if (psi[x] < m) m = psi[x];
            }
            sk[j] = m;
        }
    }
}

/* MinWise (Sec. 1): k independent permutations, min per permutation. */
int or_minwise(const uint32_t *ids, const int64_t *offsets, int64_t n,
               const uint32_t *perms, uint64_t D, uint32_t k, uint32_t *out,
               int threads) {
    minwise_ctx c;
    c.ids = ids; c.off = offsets; c.perms = perms; c.D = D; c.k = k; c.out = out;
    c.err = 0;
    run_parallel(minwise_range, &c, n, threads);
    return c.err ? -2 : 0;
}

/* ----------------------------------------------------------------------- */
/* Binomial tails (Eq. 10-11): low[m] = P(X < m), up[m] = P(X >= m)         */
/* ----------------------------------------------------------------------- */

int or_tails(uint32_t kg, uint32_t tn, uint32_t td, long double *low,
             long double *up) {
    long double *pmf;
    long double T, lT, l1T;
    uint32_t j;
    int m;
    if (td == 0 || tn > td) return -1;
    pmf = (long double *)malloc(sizeof(long double) * (kg + 1));
    T = (long double)tn / (long double)td;
    lT = logl(T);
    l1T = logl(1.0L - T);
    for (j = 0; j <= kg; ++j) {
        if (tn == 0) pmf[j] = (j == 0) ? 1.0L : 0.0L;
        else if (tn == td) pmf[j] = (j == kg) ? 1.0L : 0.0L;
        else
            pmf[j] = expl(lgammal((long double)kg + 1) - lgammal((long double)j + 1)
                          - lgammal((long double)(kg - j) + 1)
                          + (long double)j * lT + (long double)(kg - j) * l1T);
    }
    low[0] = 0.0L;
    for (m = 1; m <= (int)kg + 1; ++m) low[m] = low[m - 1] + pmf[m - 1];
    up[kg + 1] = 0.0L;
    for (m = (int)kg; m >= 0; --m) up[m] = up[m + 1] + pmf[m];
    free(pmf);
    return 0;
}

/* ----------------------------------------------------------------------- */
/* Exact tail tests (Definition 1): is P(X >= m) <= eps, is P(X < m) <= eps */
/* ----------------------------------------------------------------------- */

/* Numbers are nl little-endian 32-bit words, large enough for every value
 * below (no overflow check is needed beyond the size chosen in or_tail_ok). */
static void w_set_small(uint32_t *a, int nl, uint32_t v) {
    memset(a, 0, sizeof(uint32_t) * nl);
    a[0] = v;
}
static void w_mul_small(uint32_t *a, int nl, uint32_t m) {
    uint64_t carry = 0;
    int i;
    for (i = 0; i < nl; ++i) {
        uint64_t v = (uint64_t)a[i] * m + carry;
        a[i] = (uint32_t)v;
        carry = v >> 32;
    }
}
static void w_div_small(uint32_t *a, int nl, uint32_t d) {
    uint64_t r = 0;
    int i;
    for (i = nl - 1; i >= 0; --i) {
        uint64_t v = (r << 32) | a[i];
        a[i] = (uint32_t)(v / d);
        r = v % d;
    }
}
static void w_add(uint32_t *a, const uint32_t *b, int nl) {
    uint64_t carry = 0;
    int i;
    for (i = 0; i < nl; ++i) {
        uint64_t v = (uint64_t)a[i] + b[i] + carry;
        a[i] = (uint32_t)v;
        carry = v >> 32;
    }
}
static void w_shl(uint32_t *out, const uint32_t *a, int nl, int bits) {
    int w = bits / 32, r = bits % 32, i;
    memset(out, 0, sizeof(uint32_t) * nl);
    for (i = 0; i + w < nl; ++i) {
        out[i + w] |= a[i] << r;
        if (r && i + w + 1 < nl) out[i + w + 1] |= a[i] >> (32 - r);
    }
}
static int w_cmp(const uint32_t *a, const uint32_t *b, int nl) {
    int i;
    for (i = nl - 1; i >= 0; --i)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
}

/*
 * up_ok[m] = [P(X >= m) <= eps], low_ok[m] = [P(X < m) <= eps], m = 0..kg+1,
 * X ~ Bin(kg, tn/td).  With s = td - tn, A_i = C(kg, i) tn^i s^(kg-i) =
 * td^kg P(X = i); eps = mant 2^e2 exactly (frexp), so a tail t <= eps is
 * t td^kg 2^-e2 <= mant td^kg.  sum_i A_i = td^kg is checked against the
 * power itself.  Returns 0, or -1 on bad arguments / a failed check.
 */
int or_tail_ok(uint32_t kg, uint32_t tn, uint32_t td, double eps, uint8_t *up_ok,
               uint8_t *low_ok) {
    int bits_td = 0, nl, fe = 0, e2, rc = 0;
    uint32_t i, j, s;
    uint64_t mant;
    uint32_t *A, *tdk, *tmp, *rhs, *lhs, *up, *low;
    if (td == 0 || tn == 0 || tn > td || kg == 0 || !(eps >= 0.0)) return -1;
    s = td - tn;
    while (bits_td < 32 && (1ull << bits_td) <= td) ++bits_td;
    nl = (int)(((uint64_t)kg * bits_td + 64 + 1200) / 32 + 2);
    A = (uint32_t *)calloc((size_t)(kg + 1) * nl, sizeof(uint32_t));
    tdk = (uint32_t *)calloc(nl, sizeof(uint32_t));
    tmp = (uint32_t *)calloc(nl, sizeof(uint32_t));
    rhs = (uint32_t *)calloc(nl, sizeof(uint32_t));
    lhs = (uint32_t *)calloc(nl, sizeof(uint32_t));
    up = (uint32_t *)calloc((size_t)(kg + 2) * nl, sizeof(uint32_t));
    low = (uint32_t *)calloc((size_t)(kg + 2) * nl, sizeof(uint32_t));
    /* A_i = C(kg, i) tn^i s^(kg-i); C(kg, i) by C(kg, i-1) (kg-i+1) / i */
    w_set_small(tmp, nl, 1);
    for (i = 0; i <= kg; ++i) {
        uint32_t *a = A + (size_t)i * nl;
        if (i > 0) {
            w_mul_small(tmp, nl, kg - i + 1);
            w_div_small(tmp, nl, i);
        }
        memcpy(a, tmp, sizeof(uint32_t) * nl);
        for (j = 0; j < i; ++j) w_mul_small(a, nl, tn);
        for (j = 0; j < kg - i; ++j) w_mul_small(a, nl, s);
    }
    /* up[m] = sum_{i >= m} A_i, low[m] = sum_{i < m} A_i */
    for (i = kg + 1; i-- > 0;) {
        memcpy(up + (size_t)i * nl, up + (size_t)(i + 1) * nl, sizeof(uint32_t) * nl);
        w_add(up + (size_t)i * nl, A + (size_t)i * nl, nl);
    }
    for (i = 1; i <= kg + 1; ++i) {
        memcpy(low + (size_t)i * nl, low + (size_t)(i - 1) * nl, sizeof(uint32_t) * nl);
        w_add(low + (size_t)i * nl, A + (size_t)(i - 1) * nl, nl);
    }
    w_set_small(tdk, nl, 1);
    for (i = 0; i < kg; ++i) w_mul_small(tdk, nl, td);
    if (w_cmp(tdk, up, nl) != 0 || w_cmp(tdk, low + (size_t)(kg + 1) * nl, nl) != 0) rc = -1;
    /* rhs = mant td^kg, eps = mant 2^e2 */
    mant = (uint64_t)ldexp(frexp(eps, &fe), 53);
    e2 = fe - 53;
    if (eps == 0.0) { mant = 0; e2 = 0; }
    memcpy(rhs, tdk, sizeof(uint32_t) * nl);
    w_mul_small(rhs, nl, (uint32_t)(mant >> 32));
    w_shl(tmp, rhs, nl, 32);
    memcpy(rhs, tdk, sizeof(uint32_t) * nl);
    w_mul_small(rhs, nl, (uint32_t)mant);
    w_add(rhs, tmp, nl);
    if (e2 > 0) {
        w_shl(tmp, rhs, nl, e2);
        memcpy(rhs, tmp, sizeof(uint32_t) * nl);
    }
    for (i = 0; i <= kg + 1; ++i) {
        w_shl(lhs, up + (size_t)i * nl, nl, e2 < 0 ? -e2 : 0);
        up_ok[i] = (uint8_t)(w_cmp(lhs, rhs, nl) <= 0);
        w_shl(lhs, low + (size_t)i * nl, nl, e2 < 0 ? -e2 : 0);
        low_ok[i] = (uint8_t)(w_cmp(lhs, rhs, nl) <= 0);
    }
    free(A); free(tdk); free(tmp); free(rhs); free(lhs); free(up); free(low);
    return rc;
}

/* U = min{j : P(X >= j) <= eps}, L = max{j : P(X < j) <= eps} (for tests) */
int or_limits(uint32_t kg, uint32_t tn, uint32_t td, double eps, int64_t *U, int64_t *L) {
    uint8_t *up_ok = (uint8_t *)malloc(kg + 2), *low_ok = (uint8_t *)malloc(kg + 2);
    int64_t j;
    int rc = or_tail_ok(kg, tn, td, eps, up_ok, low_ok);
    if (rc == 0) {
        *U = kg + 1;
        for (j = (int64_t)kg + 1; j >= 0; --j) if (up_ok[j]) *U = j;
        *L = 0;
        for (j = 0; j <= (int64_t)kg + 1; ++j) if (low_ok[j]) *L = j;
    }
    free(up_ok);
    free(low_ok);
    return rc;
}

/* double-precision copy of the tails, for tests */
int or_tails_double(uint32_t kg, uint32_t tn, uint32_t td, double *low, double *up) {
    long double *l = (long double *)malloc(sizeof(long double) * (kg + 2));
    long double *u = (long double *)malloc(sizeof(long double) * (kg + 2));
    uint32_t m;
    int r = or_tails(kg, tn, td, l, u);
    for (m = 0; m < kg + 2 && r == 0; ++m) { low[m] = (double)l[m]; up[m] = (double)u[m]; }
    free(l);
    free(u);
    return r;
}

/* ----------------------------------------------------------------------- */
/* Comparison (Algorithm 1, Algorithm 2, Eq. 6)                             */
/* ----------------------------------------------------------------------- */

enum { OR_OPH_FULL = 0, OR_GOPH = 1, OR_HOPH = 2, OR_MINWISE_FULL = 3 };
enum { OR_RULE_BOTH = 0, OR_RULE_EITHER = 1, OR_RULE_NONE = 2 };
enum { OR_CONTINUE = 0, OR_ACCEPT = 1, OR_REJECT = 2 };

typedef struct {
    uint32_t mode;
    uint32_t rule;
    uint32_t k;
    uint32_t kg;
    uint32_t tn;
    uint32_t td;
    double eps;
    const uint64_t *z; /* group sizes [k/kg] (HOPH) */
    uint32_t weighting; /* 0 space-weighted, 1 Algorithm 2 as printed */
    uint32_t a, b;      /* the (a:b) split, r = a/(a+b) */
} or_query_params;

typedef struct {
    const or_query_params *p;
    uint8_t *low_ok, *up_ok; /* [kg+2]: P(X < m) <= eps, P(X >= m) <= eps */
    const uint32_t *qs, *rs;
    int64_t Q, N;
    int8_t *dec;
    uint8_t *groups;
    uint16_t *msum;
    /* per-thread accepted lists */
    int64_t **acc;
    int64_t *acc_n, *acc_cap;
    int64_t *hist; /* [threads][G+1][3] */
    uint32_t G;
    volatile int err;
} query_ctx;

static int64_t floor_div128(i128 a, i128 b) { /* b > 0 */
    i128 q = a / b;
    if ((a % b != 0) && (a < 0)) q -= 1;
    return (int64_t)q;
}
static int64_t ceil_div128(i128 a, i128 b) { return -floor_div128(-a, b); }

/* F(m) <= eps for the lower tail P(X < m) and the upper tail P(X >= m) at an
 * integer m (= ceil of the real argument); outside 0..kg+1 the tails are the
 * same as at the nearest end (0 below 0 / 1 above kg for the lower one). */
static int lower_small(const query_ctx *c, int64_t m) {
    if (m < 0) m = 0;
    if (m > (int64_t)c->p->kg + 1) m = (int64_t)c->p->kg + 1;
    return c->low_ok[m];
}
static int upper_small(const query_ctx *c, int64_t m) {
    if (m < 0) m = 0;
    if (m > (int64_t)c->p->kg + 1) m = (int64_t)c->p->kg + 1;
    return c->up_ok[m];
}

static i128 gcd128(i128 a, i128 b) {
    if (a < 0) a = -a;
    while (b) { i128 t = a % b; a = b; b = t; }
    return a;
}

/* counts over bins [b0, b1) */
static void group_counts(const uint32_t *s, const uint32_t *t, uint32_t b0, uint32_t b1,
                         int64_t *m, int64_t *e, int64_t *x) {
    uint32_t j;
    *m = *e = *x = 0;
    for (j = b0; j < b1; ++j) {
        if (s[j] == OR_EMPTY && t[j] == OR_EMPTY) (*e)++;
        else if (s[j] == OR_EMPTY || t[j] == OR_EMPTY) (*x)++;
        else if (s[j] == t[j]) (*m)++;
    }
}

static int64_t eff_bins(uint32_t rule, int64_t kg, int64_t e, int64_t x) {
    if (rule == OR_RULE_BOTH) return kg - e;
    if (rule == OR_RULE_EITHER) return kg - e - x;
    return kg;
}

/* one pair: returns decision, sets *groups and *msum */
static int compare_pair(query_ctx *c, const uint32_t *s, const uint32_t *t,
                        int *groups, int64_t *msum) {
    const or_query_params *p = c->p;
    const int64_t tn = p->tn, td = p->td, kg = p->kg;
    const int64_t n = c->G;
    int64_t m, e, x;
    if (p->mode == OR_MINWISE_FULL) {
        int64_t j, mm = 0;
        for (j = 0; j < p->k; ++j) if (s[j] != OR_EMPTY && s[j] == t[j]) mm++;
        *groups = 1; *msum = mm;
        return (mm * td >= tn * (int64_t)p->k) ? OR_ACCEPT : OR_REJECT;
    }
    if (p->mode == OR_OPH_FULL) {
        int64_t K;
        group_counts(s, t, 0, p->k, &m, &e, &x);
        K = eff_bins(p->rule, p->k, e, x);
        *groups = 1; *msum = m;
        return (K > 0 && m * td >= tn * K) ? OR_ACCEPT : OR_REJECT;
    }
    if (p->mode == OR_GOPH) {
        int64_t Mc = 0, Kc = 0, l;
        for (l = 1; l <= n; ++l) {
            i128 num, den;
            int64_t ceilm;
            group_counts(s, t, (uint32_t)((l - 1) * kg), (uint32_t)(l * kg), &m, &e, &x);
            Mc += m;
            Kc += eff_bins(p->rule, kg, e, x);
            *groups = (int)l; *msum = Mc;
            if (l == n) return (Kc > 0 && Mc * td >= tn * Kc) ? OR_ACCEPT : OR_REJECT;
            /* M_ra = (T (K_c + (n-l)k') - M_c)/(n-l) = num/den */
            num = (i128)tn * (Kc + (n - l) * kg) - (i128)td * Mc;
            den = (i128)td * (n - l);
            ceilm = ceil_div128(num, den);
            /* M_ra < M_a = T k' ?  num/den < tn kg / td */
            if (num * td < (i128)tn * kg * den) {
                if (lower_small(c, ceilm)) return OR_ACCEPT;
            } else {
                if (upper_small(c, ceilm)) return OR_REJECT;
            }
        }
        return OR_REJECT;
    }
    /* HOPH, space-weighted (or Algorithm 2's printed recursion) */
    {
        i128 Sn = 0, Sd = 1; /* S = Sn/Sd */
        i128 Pn = tn, Pd = td; /* literal: P = Pn/Pd, from P = T */
        int64_t Zd = 0, Mc = 0, l;
        for (l = 1; l <= n; ++l) {
            int64_t K, Zrem = 0, j;
            i128 num, den, g, ceilm;
            group_counts(s, t, (uint32_t)((l - 1) * kg), (uint32_t)(l * kg), &m, &e, &x);
            K = eff_bins(p->rule, kg, e, x);
            Mc += m;
            if (K > 0) {
                /* S += z m / K */
                i128 an = (i128)p->z[l - 1] * m, ad = K;
                Sn = Sn * ad + an * Sd;
                Sd = Sd * ad;
                g = gcd128(Sn, Sd);
                if (g > 1) { Sn /= g; Sd /= g; }
                Zd += (int64_t)p->z[l - 1];
            }
            *groups = (int)l; *msum = Mc;
            if (l == n)
                return (Zd > 0 && Sn * td >= (i128)tn * Zd * Sd) ? OR_ACCEPT : OR_REJECT;
            if (p->weighting == 1) {
                /* P <- (P - (m/k') r^l) / r^l with r^l = al/cl */
                i128 al = 1, cl = 1;
                for (j = 0; j < l; ++j) {
                    al *= p->a;
                    cl *= (i128)p->a + p->b;
                }
                Pn = Pn * cl * kg - (i128)m * al * Pd;
                Pd = Pd * al * kg;
                g = gcd128(Pn < 0 ? -Pn : Pn, Pd);
                if (g > 1) { Pn /= g; Pd /= g; }
                if (Pd > ((i128)1 << 60) || Pn > ((i128)1 << 60) || Pn < -((i128)1 << 60))
                    c->err = 3; /* magnitude guard */
                num = Pn;
                den = Pd;
            } else {
                for (j = l; j < n; ++j) Zrem += (int64_t)p->z[j];
                /* P_r = (T (Zd + Zrem) - S) / Zrem = num / den */
                num = (i128)tn * (Zd + Zrem) * Sd - (i128)td * Sn;
                den = (i128)td * Sd * Zrem;
                if (Sd > ((i128)1 << 60)) c->err = 3; /* magnitude guard */
            }
            ceilm = ceil_div128(num * kg, den);
            if (num * td < (i128)tn * den) { /* P_r < T */
                if (lower_small(c, (int64_t)ceilm)) return OR_ACCEPT;
            } else {
                if (upper_small(c, (int64_t)ceilm)) return OR_REJECT;
            }
        }
        return OR_REJECT;
    }
}

static void query_range(void *pv, int64_t b, int64_t e, int tid) {
    query_ctx *c = (query_ctx *)pv;
    const uint32_t k = c->p->k;
    int64_t q, r;
    for (q = b; q < e; ++q) {
        const uint32_t *s = c->qs + (size_t)q * k;
        for (r = 0; r < c->N; ++r) {
            const uint32_t *t = c->rs + (size_t)r * k;
            int groups = 0;
            int64_t msum = 0;
            int d = compare_pair(c, s, t, &groups, &msum);
            size_t idx = (size_t)q * c->N + r;
            if (c->dec) c->dec[idx] = (int8_t)d;
            if (c->groups) c->groups[idx] = (uint8_t)groups;
            if (c->msum) c->msum[idx] = (uint16_t)msum;
            if (c->hist) c->hist[((size_t)tid * (c->G + 1) + groups) * 3 + d]++;
            if (d == OR_ACCEPT) {
                if (c->acc_n[tid] == c->acc_cap[tid]) {
                    int64_t nc = c->acc_cap[tid] ? 2 * c->acc_cap[tid] : 1024;
                    c->acc[tid] = (int64_t *)realloc(c->acc[tid], sizeof(int64_t) * 4 * nc);
                    c->acc_cap[tid] = nc;
                }
                c->acc[tid][4 * c->acc_n[tid] + 0] = q;
                c->acc[tid][4 * c->acc_n[tid] + 1] = r;
                c->acc[tid][4 * c->acc_n[tid] + 2] = groups;
                c->acc[tid][4 * c->acc_n[tid] + 3] = msum;
                c->acc_n[tid]++;
            }
        }
    }
}

/*
 * Compare every (query, row) pair.  Sketches are [Q][k] and [N][k] in bin
 * order.  Optional per-pair outputs dec/groups/msum ([Q][N]); accepted pairs
 * (q, r, groups, msum) go to acc[4*i..] sorted by (q, r), at most acc_cap of
 * them; hist (nullable) receives [G+1][3] counts of (groups compared,
 * decision).  Returns the number of accepted pairs, or a negative error.
 */
int64_t or_query(const or_query_params *p, const uint32_t *qs, int64_t Q,
                 const uint32_t *rs, int64_t N, int8_t *dec, uint8_t *groups,
                 uint16_t *msum, int64_t *acc, int64_t acc_cap, int64_t *hist,
                 int threads) {
    query_ctx c;
    int t, nt;
    int64_t total = 0, i;
    uint8_t *low_ok, *up_ok;
    if (p->kg == 0 || p->k % p->kg) return -1;
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    nt = (Q < threads) ? (Q > 0 ? (int)Q : 1) : threads;
    memset(&c, 0, sizeof c);
    c.p = p;
    c.G = (p->mode == OR_GOPH || p->mode == OR_HOPH) ? p->k / p->kg : 1;
    low_ok = (uint8_t *)malloc(p->kg + 2);
    up_ok = (uint8_t *)malloc(p->kg + 2);
    if (or_tail_ok(p->kg, p->tn, p->td, p->eps, up_ok, low_ok)) {
        free(low_ok);
        free(up_ok);
        return -1;
    }
    c.low_ok = low_ok; c.up_ok = up_ok;
    c.qs = qs; c.rs = rs; c.Q = Q; c.N = N;
    c.dec = dec; c.groups = groups; c.msum = msum;
    c.acc = (int64_t **)calloc(nt, sizeof(int64_t *));
    c.acc_n = (int64_t *)calloc(nt, sizeof(int64_t));
    c.acc_cap = (int64_t *)calloc(nt, sizeof(int64_t));
    c.hist = hist ? (int64_t *)calloc((size_t)nt * (c.G + 1) * 3, sizeof(int64_t)) : 0;
    run_parallel(query_range, &c, Q, nt);
    for (t = 0; t < nt; ++t) {
        for (i = 0; i < c.acc_n[t]; ++i, ++total)
            if (total < acc_cap) memcpy(acc + 4 * total, c.acc[t] + 4 * i, sizeof(int64_t) * 4);
        free(c.acc[t]);
    }
    if (hist) {
        size_t cells = (size_t)(c.G + 1) * 3, j;
        for (j = 0; j < cells; ++j) hist[j] = 0;
        for (t = 0; t < nt; ++t)
            for (j = 0; j < cells; ++j) hist[j] += c.hist[(size_t)t * cells + j];
        free(c.hist);
    }
    free(c.acc); free(c.acc_n); free(c.acc_cap);
    free(low_ok); free(up_ok);
    if (c.err) return -3;
    return total;
}

/* Per-pair, per-group (matched, both-empty, exactly-one-empty) counts,
 * out[Q][N][G][3] as uint16 (Eq. 2-5). */
void or_pair_counts(const uint32_t *qs, int64_t Q, const uint32_t *rs, int64_t N,
                    uint32_t k, uint32_t kg, uint16_t *out) {
    int64_t q, r;
    uint32_t g, G = k / kg;
    for (q = 0; q < Q; ++q)
        for (r = 0; r < N; ++r)
            for (g = 0; g < G; ++g) {
                int64_t m, e, x;
                uint16_t *o = out + (((size_t)q * N + r) * G + g) * 3;
                group_counts(qs + (size_t)q * k, rs + (size_t)r * k, g * kg, (g + 1) * kg,
                             &m, &e, &x);
                o[0] = (uint16_t)m; o[1] = (uint16_t)e; o[2] = (uint16_t)x;
            }
}

/* ----------------------------------------------------------------------- */
/* Exact Jaccard ground truth (Sec. 3.1)                                    */
/* ----------------------------------------------------------------------- */

static int cmp_u32(const void *a, const void *b) {
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

static int64_t sorted_unique(const uint32_t *src, int64_t n, uint32_t *dst) {
    int64_t i, m = 0;
    memcpy(dst, src, sizeof(uint32_t) * (size_t)n);
    qsort(dst, (size_t)n, sizeof(uint32_t), cmp_u32);
    for (i = 0; i < n; ++i)
        if (m == 0 || dst[m - 1] != dst[i]) dst[m++] = dst[i];
    return m;
}

typedef struct {
    const uint32_t *aid, *bid;
    const int64_t *aoff, *boff;
    const int64_t *pa, *pb;
    int64_t *inter, *uni;
} jac_ctx;

static void jac_range(void *pv, int64_t b, int64_t e, int tid) {
    jac_ctx *c = (jac_ctx *)pv;
    int64_t i;
    (void)tid;
    for (i = b; i < e; ++i) {
        int64_t ia = c->pa[i], ib = c->pb[i];
        int64_t na = c->aoff[ia + 1] - c->aoff[ia], nb = c->boff[ib + 1] - c->boff[ib];
        uint32_t *A = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(na + 1));
        uint32_t *B = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nb + 1));
        int64_t ua = sorted_unique(c->aid + c->aoff[ia], na, A);
        int64_t ub = sorted_unique(c->bid + c->boff[ib], nb, B);
        int64_t x = 0, y = 0, both = 0;
        while (x < ua && y < ub) {
            if (A[x] == B[y]) { both++; x++; y++; }
            else if (A[x] < B[y]) x++;
            else y++;
        }
        c->inter[i] = both;
        c->uni[i] = ua + ub - both;
        free(A);
        free(B);
    }
}

/* |A n B| and |A u B| (distinct elements) for n_pairs pairs (A = set pa[i]
 * of collection a, B = set pb[i] of collection b). */
void or_jaccard_pairs(const uint32_t *aid, const int64_t *aoff, const uint32_t *bid,
                      const int64_t *boff, const int64_t *pa, const int64_t *pb,
                      int64_t n_pairs, int64_t *inter, int64_t *uni, int threads) {
    jac_ctx c;
    c.aid = aid; c.bid = bid; c.aoff = aoff; c.boff = boff; c.pa = pa; c.pb = pb;
    c.inter = inter; c.uni = uni;
    run_parallel(jac_range, &c, n_pairs, threads);
}
