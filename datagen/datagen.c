/*
 * datagen.c -- seeded synthetic inputs for forest classification.
 *
 * This module produces the two inputs of the classification path that the
 * paper takes as given (Section III starts from a forest that has already
 * been trained): observation matrices and a trained random forest.  It contains no
 * part of the packing or classification method itself; both the CPU oracle
 * and the GPU library consume what it writes.
 *
 * Randomness: SplitMix64 (Steele, Lea & Flood, 2014) seeds xoshiro256**
 * (Blackman & Vigna, 2018).  Every (seed, purpose, index) triple owns an
 * independent stream, so results do not depend on thread count or order.
 * Normals use the Box-Muller transform (Box & Muller, 1958).
 *
 * Trainer: CART random forest (Breiman 2001), as the paper's forests are
 * (Section IV-C: Gini splits, trees grown to maximum depth, leaves of a single
 * observation).  Details the paper leaves open are fixed here:
 *   - bootstrap of n draws with replacement, multiplicities kept as weights;
 *   - mtry = floor(sqrt(d)) features per node, drawn without replacement by a
 *     partial Fisher-Yates shuffle; if none of them has two distinct values on
 *     the node, further features of the same permutation are drawn until one
 *     does (needed to grow to purity);
 *   - thresholds sit between consecutive distinct values a < b at the float
 *     midpoint, falling back to a when rounding lands on b; x <= t goes left;
 *   - the split maximises sum_c L_c^2/W_L + sum_c R_c^2/W_R (equivalent to the
 *     weighted Gini decrease), compared exactly with 128-bit integers; ties keep
 *     the earlier feature in draw order, then the smaller threshold;
 *   - a node is a leaf when pure or when no feature can split it; its class is
 *     the weighted majority, lowest class index on ties;
 *   - cardinality = in-bag count with multiplicity reaching the node;
 *   - node ids are pre-order creation order within a tree.
 *
 * Compiled without -ffast-math and with -ffp-contract=off.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ PRNG */

typedef struct { uint64_t s[4]; } dg_rng;

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t mix64(uint64_t z) {
    uint64_t x = z;
    return splitmix64_next(&x);
}

void dg_rng_init(dg_rng *r, uint64_t seed, uint64_t purpose, uint64_t index) {
    uint64_t k = mix64(seed);
    k = mix64(k ^ mix64(purpose * 0xD1B54A32D192ED03ULL + 1));
    k = mix64(k ^ mix64(index * 0x8CB92BA72F3D8DD7ULL + 7));
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&k);
}

uint64_t dg_next(dg_rng *r) {
    uint64_t *s = r->s;
    const uint64_t result = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

/* uniform on [0, 1) with 53 random bits */
static inline double dg_uniform(dg_rng *r) { return (double)(dg_next(r) >> 11) * 0x1.0p-53; }
/* uniform on (0, 1] */
static inline double dg_uniform_pos(dg_rng *r) { return 1.0 - dg_uniform(r); }
/* integer in [0, n): multiply-shift */
static inline uint64_t dg_bounded(dg_rng *r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)dg_next(r) * n) >> 64);
}
/* standard normal, Box-Muller (one of the pair is used) */
static inline double dg_normal(dg_rng *r) {
    const double u1 = dg_uniform_pos(r);
    const double u2 = dg_uniform(r);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* exported for tests of the generator itself */
uint64_t dg_stream_first(uint64_t seed, uint64_t purpose, uint64_t index) {
    dg_rng r;
    dg_rng_init(&r, seed, purpose, index);
    return dg_next(&r);
}

/* xoshiro256** reference check: with state {1,2,3,4} the first outputs are
 * fixed by the published algorithm; tests compare against them. */
void dg_xoshiro_from_state(const uint64_t state[4], int n, uint64_t *out) {
    dg_rng r;
    memcpy(r.s, state, sizeof r.s);
    for (int i = 0; i < n; ++i) out[i] = dg_next(&r);
}

enum {
    PURPOSE_PARAMS = 1,  /* per-dataset parameters: means, block stats, weights */
    PURPOSE_ROWS = 2,    /* observation rows, index = split * 2^32 + chunk */
    PURPOSE_TREE = 3,    /* trainer: bootstrap and feature draws of one tree */
};

#define DG_CHUNK 65536

/* ------------------------------------------------------- parallel helper */

typedef void (*dg_chunk_fn)(void *ctx, int64_t chunk);
typedef struct { dg_chunk_fn fn; void *ctx; int64_t n_chunks; int64_t next; pthread_mutex_t mu; } dg_pool;

static void *dg_pool_worker(void *arg) {
    dg_pool *p = (dg_pool *)arg;
    for (;;) {
        pthread_mutex_lock(&p->mu);
        int64_t c = p->next++;
        pthread_mutex_unlock(&p->mu);
        if (c >= p->n_chunks) break;
        p->fn(p->ctx, c);
    }
    return NULL;
}

static void dg_parallel(dg_chunk_fn fn, void *ctx, int64_t n_chunks, int n_threads) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    if (n_threads > n_chunks) n_threads = (int)(n_chunks > 0 ? n_chunks : 1);
    dg_pool p = {fn, ctx, n_chunks, 0, PTHREAD_MUTEX_INITIALIZER};
    if (n_threads == 1) {
        for (int64_t c = 0; c < n_chunks; ++c) fn(ctx, c);
        return;
    }
    pthread_t th[256];
    for (int i = 0; i < n_threads; ++i) pthread_create(&th[i], NULL, dg_pool_worker, &p);
    for (int i = 0; i < n_threads; ++i) pthread_join(th[i], NULL);
}

/* ------------------------------------------------------------ generators */

/* Gaussian mixture: class means mu_c ~ U[lo, hi]^d from the parameter stream;
 * y ~ uniform over classes; x = mu_y + N(0, I). */
typedef struct {
    uint64_t seed; int64_t n; int32_t d, C; uint32_t split; const double *mu;
    float *X; int32_t *y;
} mix_ctx;

static void mix_chunk(void *vc, int64_t chunk) {
    mix_ctx *c = (mix_ctx *)vc;
    dg_rng r;
    dg_rng_init(&r, c->seed, PURPOSE_ROWS, ((uint64_t)c->split << 32) | (uint64_t)chunk);
    int64_t a = chunk * DG_CHUNK, b = a + DG_CHUNK;
    if (b > c->n) b = c->n;
    for (int64_t i = a; i < b; ++i) {
        int32_t k = (int32_t)dg_bounded(&r, (uint64_t)c->C);
        c->y[i] = k;
        for (int32_t f = 0; f < c->d; ++f)
            c->X[i * c->d + f] = (float)(c->mu[(int64_t)k * c->d + f] + dg_normal(&r));
    }
}

int dg_gen_mixture(uint64_t seed, int32_t C, int32_t d, double lo, double hi, int64_t n,
                   uint32_t split, float *X, int32_t *y, int n_threads) {
    if (C < 1 || d < 1 || n < 0) return -1;
    double *mu = (double *)malloc(sizeof(double) * (size_t)C * (size_t)d);
    if (!mu) return -2;
    dg_rng r;
    dg_rng_init(&r, seed, PURPOSE_PARAMS, 0);
    for (int64_t i = 0; i < (int64_t)C * d; ++i) mu[i] = lo + (hi - lo) * dg_uniform(&r);
    mix_ctx c = {seed, n, d, C, split, mu, X, y};
    dg_parallel(mix_chunk, &c, (n + DG_CHUNK - 1) / DG_CHUNK, n_threads);
    free(mu);
    return 0;
}

/* Image-shaped rows: 28x28 pixels in 16 blocks of 7x7.  Per (class, block):
 * zero probability p ~ U(0.65, 0.95) rescaled so the mean over all (class,
 * block) pairs is 0.8, and an exponent k ~ U(1/3, 3).  A pixel is 0 with
 * probability p, else u^k with u ~ U(0, 1].  Classes are balanced: y = i mod 10. */
#define IMG_C 10
#define IMG_D 784
#define IMG_BLOCKS 16

typedef struct { uint64_t seed; int64_t n; uint32_t split; double p[IMG_C][IMG_BLOCKS]; double k[IMG_C][IMG_BLOCKS]; float *X; int32_t *y; } img_ctx;

static void img_chunk(void *vc, int64_t chunk) {
    img_ctx *c = (img_ctx *)vc;
    dg_rng r;
    dg_rng_init(&r, c->seed, PURPOSE_ROWS, ((uint64_t)c->split << 32) | (uint64_t)chunk);
    int64_t a = chunk * DG_CHUNK, b = a + DG_CHUNK;
    if (b > c->n) b = c->n;
    for (int64_t i = a; i < b; ++i) {
        int32_t cls = (int32_t)(i % IMG_C);
        c->y[i] = cls;
        for (int f = 0; f < IMG_D; ++f) {
            int row = f / 28, col = f % 28;
            int blk = (row / 7) * 4 + (col / 7);
            double u0 = dg_uniform(&r);
            double u1 = dg_uniform_pos(&r);
            float v = 0.0f;
            if (u0 >= c->p[cls][blk]) v = (float)pow(u1, c->k[cls][blk]);
            c->X[i * IMG_D + f] = v;
        }
    }
}

int dg_gen_image(uint64_t seed, int64_t n, uint32_t split, float *X, int32_t *y, int n_threads) {
    img_ctx *c = (img_ctx *)calloc(1, sizeof(img_ctx));
    if (!c) return -2;
    c->seed = seed; c->n = n; c->split = split; c->X = X; c->y = y;
    dg_rng r;
    dg_rng_init(&r, seed, PURPOSE_PARAMS, 0);
    double mean = 0;
    for (int k = 0; k < IMG_C; ++k)
        for (int b = 0; b < IMG_BLOCKS; ++b) {
            c->p[k][b] = 0.65 + 0.30 * dg_uniform(&r);
            c->k[k][b] = 1.0 / 3.0 + (3.0 - 1.0 / 3.0) * dg_uniform(&r);
            mean += c->p[k][b];
        }
    mean /= (double)(IMG_C * IMG_BLOCKS);
    for (int k = 0; k < IMG_C; ++k)
        for (int b = 0; b < IMG_BLOCKS; ++b) {
            double p = c->p[k][b] * 0.8 / mean;
            c->p[k][b] = p > 0.99 ? 0.99 : p;
        }
    dg_parallel(img_chunk, c, (n + DG_CHUNK - 1) / DG_CHUNK, n_threads);
    free(c);
    return 0;
}

/* Logistic rows: 21 N(0,1) features and 7 LogNormal(0,1) features; z is x with
 * log applied to the log-normal ones.  y ~ Bernoulli(sigmoid(s * (w.z +
 * sum_{(i,j) in P} v_ij z_i z_j))) with w ~ N(0, 1/28), 28 random pairs i != j,
 * v ~ N(0, 0.25).  The scale s sets the label noise and so the tree size. */
#define LOG_D 28
#define LOG_NNORM 21
#define LOG_PAIRS 28

typedef struct { uint64_t seed; int64_t n; uint32_t split; double s; double w[LOG_D]; int pi[LOG_PAIRS], pj[LOG_PAIRS]; double v[LOG_PAIRS]; float *X; int32_t *y; double *yr; double noise; } log_ctx;

static void log_chunk(void *vc, int64_t chunk) {
    log_ctx *c = (log_ctx *)vc;
    dg_rng r;
    dg_rng_init(&r, c->seed, PURPOSE_ROWS, ((uint64_t)c->split << 32) | (uint64_t)chunk);
    int64_t a = chunk * DG_CHUNK, b = a + DG_CHUNK;
    if (b > c->n) b = c->n;
    double z[LOG_D];
    for (int64_t i = a; i < b; ++i) {
        double logit = 0;
        for (int f = 0; f < LOG_D; ++f) {
            z[f] = dg_normal(&r);
            c->X[i * LOG_D + f] = (float)(f < LOG_NNORM ? z[f] : exp(z[f]));
            logit += c->w[f] * z[f];
        }
        for (int q = 0; q < LOG_PAIRS; ++q) logit += c->v[q] * z[c->pi[q]] * z[c->pj[q]];
        if (c->yr) {  /* regression target: the score plus Gaussian noise */
            c->yr[i] = c->s * logit + c->noise * dg_normal(&r);
            continue;
        }
        double p = 1.0 / (1.0 + exp(-c->s * logit));
        c->y[i] = dg_uniform(&r) < p ? 1 : 0;
    }
}

static int gen_logistic_like(uint64_t seed, int64_t n, uint32_t split, double scale, float *X, int32_t *y,
                             double *yr, double noise, int n_threads) {
    log_ctx *c = (log_ctx *)calloc(1, sizeof(log_ctx));
    if (!c) return -2;
    c->seed = seed; c->n = n; c->split = split; c->s = scale; c->X = X; c->y = y; c->yr = yr; c->noise = noise;
    dg_rng r;
    dg_rng_init(&r, seed, PURPOSE_PARAMS, 0);
    for (int f = 0; f < LOG_D; ++f) c->w[f] = dg_normal(&r) * sqrt(1.0 / LOG_D);
    for (int q = 0; q < LOG_PAIRS; ++q) {
        int i = (int)dg_bounded(&r, LOG_D);
        int j = (int)dg_bounded(&r, LOG_D - 1);
        if (j >= i) ++j;
        c->pi[q] = i; c->pj[q] = j;
        c->v[q] = dg_normal(&r) * 0.5;
    }
    dg_parallel(log_chunk, c, (n + DG_CHUNK - 1) / DG_CHUNK, n_threads);
    free(c);
    return 0;
}

int dg_gen_logistic(uint64_t seed, int64_t n, uint32_t split, double scale, float *X, int32_t *y, int n_threads) {
    return gen_logistic_like(seed, n, split, scale, X, y, NULL, 0.0, n_threads);
}

/* Regression rows: the features of the logistic generator and a real target
 * y = scale * (w.z + sum v_ij z_i z_j) + noise * N(0, 1). */
int dg_gen_regression(uint64_t seed, int64_t n, uint32_t split, double scale, double noise, float *X, double *y,
                      int n_threads) {
    return gen_logistic_like(seed, n, split, scale, X, NULL, y, noise, n_threads);
}

/* --------------------------------------------------------------- trainer */

typedef struct {
    int32_t *left, *right, *feature, *leaf_class;
    float *threshold;
    float *value;             /* leaf value (regression and boosted trees; 0 elsewhere) */
    int64_t *card;
    int64_t n_nodes, cap;
    int32_t depth;            /* maximum node depth (root = 0) */
    int64_t n_boot;           /* bootstrap size (sum of leaf cardinalities) */
    int oom;
} dg_tree;

typedef struct {
    int32_t n_trees, n_features, n_classes;
    dg_tree *trees;
} dg_forest;

typedef struct {
    const float *X; const int32_t *y; int64_t n; int32_t d, C, mtry; uint64_t seed;
    dg_forest *F;
} train_ctx;

/* per-thread scratch for one tree */
typedef struct {
    int32_t *samp;      /* distinct in-bag sample ids, partitioned per node */
    int64_t *w;         /* multiplicity per sample id (length n) */
    int32_t *tmp;       /* partition buffer */
    uint32_t *key, *key2;
    int32_t *pay, *pay2;
    int32_t *perm;      /* feature permutation */
    int64_t *cnt_node, *cnt_l, *cnt_r;
    int64_t *cnt_stack; /* per-depth node class counts */
    int64_t stack_cap;
    dg_rng rng;
} tree_ws;

static inline uint32_t float_key(float v) {
    if (v == 0.0f) v = 0.0f; /* -0 and +0 compare equal: give them one key */
    uint32_t u;
    memcpy(&u, &v, 4);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
static inline float key_float(uint32_t k) {
    uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
    float v;
    memcpy(&v, &u, 4);
    return v;
}

/* sort (key, payload) ascending by key; ties keep input order (stable) */
static void sort_pairs(uint32_t *k, int32_t *p, uint32_t *k2, int32_t *p2, int64_t m) {
    if (m < 48) {
        for (int64_t i = 1; i < m; ++i) {
            uint32_t kk = k[i]; int32_t pp = p[i];
            int64_t j = i - 1;
            while (j >= 0 && k[j] > kk) { k[j + 1] = k[j]; p[j + 1] = p[j]; --j; }
            k[j + 1] = kk; p[j + 1] = pp;
        }
        return;
    }
    uint32_t *src_k = k, *dst_k = k2;
    int32_t *src_p = p, *dst_p = p2;
    for (int shift = 0; shift < 32; shift += 8) {
        int64_t hist[257];
        memset(hist, 0, sizeof hist);
        for (int64_t i = 0; i < m; ++i) hist[((src_k[i] >> shift) & 255u) + 1]++;
        if (hist[((src_k[0] >> shift) & 255u) + 1] == m) continue; /* one bucket: skip pass */
        for (int b = 0; b < 256; ++b) hist[b + 1] += hist[b];
        for (int64_t i = 0; i < m; ++i) {
            int64_t pos = hist[(src_k[i] >> shift) & 255u]++;
            dst_k[pos] = src_k[i];
            dst_p[pos] = src_p[i];
        }
        uint32_t *tk = src_k; src_k = dst_k; dst_k = tk;
        int32_t *tp = src_p; src_p = dst_p; dst_p = tp;
    }
    if (src_k != k) {
        memcpy(k, src_k, sizeof(uint32_t) * (size_t)m);
        memcpy(p, src_p, sizeof(int32_t) * (size_t)m);
    }
}

static int64_t tree_push(dg_tree *t) {
    if (t->n_nodes == t->cap) {
        int64_t nc = t->cap ? t->cap * 2 : 1024;
        int32_t *l = realloc(t->left, sizeof(int32_t) * nc), *r2;
        if (!l) { t->oom = 1; return -1; }
        t->left = l;
        r2 = realloc(t->right, sizeof(int32_t) * nc); if (!r2) { t->oom = 1; return -1; } t->right = r2;
        r2 = realloc(t->feature, sizeof(int32_t) * nc); if (!r2) { t->oom = 1; return -1; } t->feature = r2;
        r2 = realloc(t->leaf_class, sizeof(int32_t) * nc); if (!r2) { t->oom = 1; return -1; } t->leaf_class = r2;
        float *th = realloc(t->threshold, sizeof(float) * nc); if (!th) { t->oom = 1; return -1; } t->threshold = th;
        th = realloc(t->value, sizeof(float) * nc); if (!th) { t->oom = 1; return -1; } t->value = th;
        int64_t *cd = realloc(t->card, sizeof(int64_t) * nc); if (!cd) { t->oom = 1; return -1; } t->card = cd;
        t->cap = nc;
    }
    return t->n_nodes++;
}

/* score of a split as the rational num/den, num = A_L*W_R + A_R*W_L, den = W_L*W_R */
static inline int score_better(int64_t num, int64_t den, int64_t bnum, int64_t bden) {
    return (__int128)num * (__int128)bden > (__int128)bnum * (__int128)den;
}

/* Evaluate the best threshold of feature f on samples samp[lo:hi].
 * Returns 1 if the feature has two distinct values there. */
static int best_split_feature(const train_ctx *c, tree_ws *ws, int64_t lo, int64_t hi, int32_t f,
                              const int64_t *cnt_node, int64_t W, int64_t *out_num, int64_t *out_den,
                              float *out_thr) {
    const int64_t m = hi - lo;
    const int32_t C = c->C;
    for (int64_t i = 0; i < m; ++i) {
        int32_t s = ws->samp[lo + i];
        ws->key[i] = float_key(c->X[(int64_t)s * c->d + f]);
        ws->pay[i] = s;
    }
    sort_pairs(ws->key, ws->pay, ws->key2, ws->pay2, m);
    if (ws->key[0] == ws->key[m - 1]) return 0;
    int64_t *cl = ws->cnt_l, *cr = ws->cnt_r;
    memset(cl, 0, sizeof(int64_t) * C);
    memcpy(cr, cnt_node, sizeof(int64_t) * C);
    int64_t AL = 0, AR = 0, WL = 0, WR = W;
    for (int32_t k = 0; k < C; ++k) AR += cr[k] * cr[k];
    int64_t bnum = -1, bden = 1;
    float bthr = 0.0f;
    for (int64_t i = 0; i + 1 < m; ++i) {
        int32_t s = ws->pay[i];
        int64_t wi = ws->w[s];
        int32_t k = c->y[s];
        AL += 2 * cl[k] * wi + wi * wi;
        AR -= 2 * cr[k] * wi - wi * wi;
        cl[k] += wi; cr[k] -= wi;
        WL += wi; WR -= wi;
        if (ws->key[i] != ws->key[i + 1]) {
            int64_t num = AL * WR + AR * WL, den = WL * WR;
            if (bnum < 0 || score_better(num, den, bnum, bden)) {
                float a = key_float(ws->key[i]), b = key_float(ws->key[i + 1]);
                float t = (float)((double)a + ((double)b - (double)a) * 0.5);
                if (!(t >= a && t < b)) t = a;
                bnum = num; bden = den; bthr = t;
            }
        }
    }
    *out_num = bnum; *out_den = bden; *out_thr = bthr;
    return 1;
}

static int64_t grow(const train_ctx *c, tree_ws *ws, dg_tree *t, int64_t lo, int64_t hi, int32_t depth) {
    int64_t id = tree_push(t);
    if (id < 0) return -1;
    if (depth > t->depth) t->depth = depth;
    const int32_t C = c->C, d = c->d;
    if ((int64_t)(depth + 1) * C > ws->stack_cap) {
        int64_t nc = ws->stack_cap * 2;
        int64_t *p = realloc(ws->cnt_stack, sizeof(int64_t) * nc);
        if (!p) { t->oom = 1; return -1; }
        ws->cnt_stack = p; ws->stack_cap = nc;
    }
    int64_t *cnt = ws->cnt_stack + (int64_t)depth * C;
    memset(cnt, 0, sizeof(int64_t) * C);
    int64_t W = 0;
    for (int64_t i = lo; i < hi; ++i) {
        int32_t s = ws->samp[i];
        cnt[c->y[s]] += ws->w[s];
        W += ws->w[s];
    }
    t->card[id] = W;
    int32_t nz = 0, maj = 0;
    for (int32_t k = 0; k < C; ++k) {
        if (cnt[k] > 0) ++nz;
        if (cnt[k] > cnt[maj]) maj = k;
    }
    t->left[id] = -1; t->right[id] = -1; t->feature[id] = -1; t->threshold[id] = 0.0f; t->leaf_class[id] = maj;
    t->value[id] = 0.0f;
    if (nz <= 1) return id;

    /* feature draws: partial Fisher-Yates, continued until a feature splits */
    for (int32_t f = 0; f < d; ++f) ws->perm[f] = f;
    int32_t bf = -1;
    int64_t bnum = -1, bden = 1;
    float bthr = 0.0f;
    for (int32_t i = 0; i < d; ++i) {
        int32_t j = i + (int32_t)dg_bounded(&ws->rng, (uint64_t)(d - i));
        int32_t tmpf = ws->perm[i]; ws->perm[i] = ws->perm[j]; ws->perm[j] = tmpf;
        int32_t f = ws->perm[i];
        int64_t num, den; float thr;
        if (best_split_feature(c, ws, lo, hi, f, cnt, W, &num, &den, &thr)) {
            if (bf < 0 || score_better(num, den, bnum, bden)) { bf = f; bnum = num; bden = den; bthr = thr; }
        }
        if (i + 1 >= c->mtry && bf >= 0) break;
    }
    if (bf < 0) return id; /* no feature separates the node: impure leaf */

    /* stable partition: x <= thr first */
    int64_t nl = 0;
    for (int64_t i = lo; i < hi; ++i) {
        int32_t s = ws->samp[i];
        if (c->X[(int64_t)s * d + bf] <= bthr) ws->samp[lo + nl++] = s; else ws->tmp[i - lo - nl] = s;
    }
    memcpy(ws->samp + lo + nl, ws->tmp, sizeof(int32_t) * (size_t)(hi - lo - nl));
    t->feature[id] = bf;
    t->threshold[id] = bthr;
    t->leaf_class[id] = -1;
    int64_t l = grow(c, ws, t, lo, lo + nl, depth + 1);
    if (l < 0) return -1;
    int64_t r = grow(c, ws, t, lo + nl, hi, depth + 1);
    if (r < 0) return -1;
    t->left[id] = (int32_t)l;
    t->right[id] = (int32_t)r;
    return id;
}

typedef struct { train_ctx *c; int64_t next; pthread_mutex_t mu; int fail; } train_pool;

static void train_one(train_ctx *c, tree_ws *ws, int32_t ti) {
    dg_tree *t = &c->F->trees[ti];
    dg_rng_init(&ws->rng, c->seed, PURPOSE_TREE, (uint64_t)ti);
    memset(ws->w, 0, sizeof(int64_t) * (size_t)c->n);
    for (int64_t i = 0; i < c->n; ++i) ws->w[dg_bounded(&ws->rng, (uint64_t)c->n)]++;
    int64_t m = 0;
    for (int64_t i = 0; i < c->n; ++i)
        if (ws->w[i]) ws->samp[m++] = (int32_t)i;
    t->n_boot = c->n;
    grow(c, ws, t, 0, m, 0);
}

static void *train_worker(void *arg) {
    train_pool *p = (train_pool *)arg;
    train_ctx *c = p->c;
    tree_ws ws;
    memset(&ws, 0, sizeof ws);
    size_t n = (size_t)c->n;
    ws.samp = malloc(sizeof(int32_t) * n);
    ws.w = malloc(sizeof(int64_t) * n);
    ws.tmp = malloc(sizeof(int32_t) * n);
    ws.key = malloc(sizeof(uint32_t) * n);
    ws.key2 = malloc(sizeof(uint32_t) * n);
    ws.pay = malloc(sizeof(int32_t) * n);
    ws.pay2 = malloc(sizeof(int32_t) * n);
    ws.perm = malloc(sizeof(int32_t) * (size_t)c->d);
    ws.cnt_node = malloc(sizeof(int64_t) * (size_t)c->C);
    ws.cnt_l = malloc(sizeof(int64_t) * (size_t)c->C);
    ws.cnt_r = malloc(sizeof(int64_t) * (size_t)c->C);
    ws.stack_cap = (int64_t)c->C * 128;
    ws.cnt_stack = malloc(sizeof(int64_t) * (size_t)ws.stack_cap);
    int ok = ws.samp && ws.w && ws.tmp && ws.key && ws.key2 && ws.pay && ws.pay2 && ws.perm &&
             ws.cnt_node && ws.cnt_l && ws.cnt_r && ws.cnt_stack;
    for (;;) {
        pthread_mutex_lock(&p->mu);
        int64_t ti = p->next++;
        if (!ok) p->fail = 1;
        pthread_mutex_unlock(&p->mu);
        if (!ok || ti >= c->F->n_trees) break;
        train_one(c, &ws, (int32_t)ti);
        if (c->F->trees[ti].oom) { pthread_mutex_lock(&p->mu); p->fail = 1; pthread_mutex_unlock(&p->mu); }
    }
    free(ws.samp); free(ws.w); free(ws.tmp); free(ws.key); free(ws.key2); free(ws.pay); free(ws.pay2);
    free(ws.perm); free(ws.cnt_node); free(ws.cnt_l); free(ws.cnt_r); free(ws.cnt_stack);
    return NULL;
}

void dg_forest_free(dg_forest *F) {
    if (!F) return;
    for (int32_t t = 0; t < F->n_trees; ++t) {
        dg_tree *tr = &F->trees[t];
        free(tr->left); free(tr->right); free(tr->feature); free(tr->leaf_class); free(tr->threshold); free(tr->card);
        free(tr->value);
    }
    free(F->trees);
    free(F);
}

/* Train a forest.  Returns NULL on bad arguments or allocation failure. */
dg_forest *dg_train(const float *X, const int32_t *y, int64_t n, int32_t d, int32_t C, int32_t n_trees,
                    int32_t mtry, uint64_t seed, int n_threads) {
    if (n < 1 || n > INT32_MAX || d < 1 || C < 1 || n_trees < 1 || mtry < 1) return NULL;
    for (int64_t i = 0; i < n; ++i)
        if (y[i] < 0 || y[i] >= C) return NULL;
    dg_forest *F = calloc(1, sizeof(dg_forest));
    if (!F) return NULL;
    F->n_trees = n_trees; F->n_features = d; F->n_classes = C;
    F->trees = calloc((size_t)n_trees, sizeof(dg_tree));
    if (!F->trees) { free(F); return NULL; }
    train_ctx c = {X, y, n, d, C, mtry > d ? d : mtry, seed, F};
    train_pool p = {&c, 0, PTHREAD_MUTEX_INITIALIZER, 0};
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n_trees) n_threads = n_trees;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    for (int i = 0; i < n_threads; ++i) pthread_create(&th[i], NULL, train_worker, &p);
    for (int i = 0; i < n_threads; ++i) pthread_join(th[i], NULL);
    if (p.fail) { dg_forest_free(F); return NULL; }
    return F;
}

int64_t dg_forest_total_nodes(const dg_forest *F) {
    int64_t s = 0;
    for (int32_t t = 0; t < F->n_trees; ++t) s += F->trees[t].n_nodes;
    return s;
}

int32_t dg_forest_n_trees(const dg_forest *F) { return F->n_trees; }

/* Copy the forest out as flat arrays; node_begin has n_trees+1 entries. */
void dg_forest_export(const dg_forest *F, int64_t *node_begin, int32_t *left, int32_t *right, int32_t *feature,
                      float *threshold, int32_t *leaf_class, int64_t *card, int32_t *tree_depth) {
    int64_t off = 0;
    for (int32_t t = 0; t < F->n_trees; ++t) {
        const dg_tree *tr = &F->trees[t];
        node_begin[t] = off;
        size_t m = (size_t)tr->n_nodes;
        memcpy(left + off, tr->left, 4 * m);
        memcpy(right + off, tr->right, 4 * m);
        memcpy(feature + off, tr->feature, 4 * m);
        memcpy(threshold + off, tr->threshold, 4 * m);
        memcpy(leaf_class + off, tr->leaf_class, 4 * m);
        memcpy(card + off, tr->card, 8 * m);
        if (tree_depth) tree_depth[t] = tr->depth;
        off += tr->n_nodes;
    }
    node_begin[F->n_trees] = off;
}

/* bootstrap multiplicities of tree t (length n), for tests of the trainer */
void dg_bootstrap_weights(uint64_t seed, int32_t tree, int64_t n, int64_t *w) {
    dg_rng r;
    dg_rng_init(&r, seed, PURPOSE_TREE, (uint64_t)tree);
    memset(w, 0, sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) w[dg_bounded(&r, (uint64_t)n)]++;
}

/* ------------------------------------------------------ regression trainer */
/* Least-squares regression trees (CART) in two forest forms, for forests with
 * real leaf values:
 *   random forest (Breiman 2001): each tree on a bootstrap of the rows with
 *     multiplicities as weights and mtry features per node (draws continued
 *     as in the classifier); a node is a leaf when its targets are all equal,
 *     when it holds less than 2*min_leaf weight, or at max_depth (0 = no
 *     limit); leaf value = weighted mean of the node's targets; the forest
 *     predicts the mean of its trees;
 *   gradient boosting with squared loss (Friedman 2001): F_0 = mean(y); round
 *     m fits a tree of depth <= max_depth to the residuals y - F_{m-1}(x) of
 *     all rows (weight 1); leaf value = eta * mean residual; the forest
 *     predicts F_0 + the sum of its trees.
 * Split: maximise S_L^2/W_L + S_R^2/W_R (S = weighted target sum, W = weight;
 * the squared-error decrease up to a constant) in double precision, samples
 * accumulated in ascending feature order; both sides must hold weight >=
 * min_leaf; ties keep the earlier feature in draw order, then the smaller
 * threshold.  Thresholds as in the classifier.  A leaf value is rounded to
 * float once; boosting adds that float value to the rows' running score. */

typedef struct {
    const float *X; const double *y; int64_t n; int32_t d, mtry, max_depth; int64_t min_leaf; uint64_t seed;
    double eta; dg_forest *F;
    const double *target;  /* what the current tree fits: y (forest) or the residuals (boosting) */
    double *score;         /* boosting: F(x_i) of the training rows, updated at each leaf */
} reg_ctx;

typedef struct {
    int32_t *samp, *tmp, *pay, *pay2, *perm;
    int64_t *w;
    uint32_t *key, *key2;
    dg_rng rng;
} reg_ws;

static int reg_ws_alloc(reg_ws *ws, int64_t n, int32_t d) {
    memset(ws, 0, sizeof *ws);
    ws->samp = malloc(sizeof(int32_t) * (size_t)n);
    ws->tmp = malloc(sizeof(int32_t) * (size_t)n);
    ws->pay = malloc(sizeof(int32_t) * (size_t)n);
    ws->pay2 = malloc(sizeof(int32_t) * (size_t)n);
    ws->perm = malloc(sizeof(int32_t) * (size_t)d);
    ws->w = malloc(sizeof(int64_t) * (size_t)n);
    ws->key = malloc(sizeof(uint32_t) * (size_t)n);
    ws->key2 = malloc(sizeof(uint32_t) * (size_t)n);
    return ws->samp && ws->tmp && ws->pay && ws->pay2 && ws->perm && ws->w && ws->key && ws->key2;
}

static void reg_ws_free(reg_ws *ws) {
    free(ws->samp); free(ws->tmp); free(ws->pay); free(ws->pay2); free(ws->perm); free(ws->w);
    free(ws->key); free(ws->key2);
}

/* Best threshold of feature f on samp[lo:hi]; returns 1 if a split with both
 * sides >= min_leaf exists. */
static int best_split_reg(const reg_ctx *c, reg_ws *ws, int64_t lo, int64_t hi, int32_t f, double S, int64_t W,
                          double *out_score, float *out_thr) {
    const int64_t m = hi - lo;
    for (int64_t i = 0; i < m; ++i) {
        int32_t s = ws->samp[lo + i];
        ws->key[i] = float_key(c->X[(int64_t)s * c->d + f]);
        ws->pay[i] = s;
    }
    sort_pairs(ws->key, ws->pay, ws->key2, ws->pay2, m);
    if (ws->key[0] == ws->key[m - 1]) return 0;
    double SL = 0.0, best = 0.0;
    int64_t WL = 0;
    int found = 0;
    float bthr = 0.0f;
    for (int64_t i = 0; i + 1 < m; ++i) {
        int32_t s = ws->pay[i];
        int64_t wi = ws->w[s];
        SL += (double)wi * c->target[s];
        WL += wi;
        if (ws->key[i] == ws->key[i + 1]) continue;
        const int64_t WR = W - WL;
        if (WL < c->min_leaf || WR < c->min_leaf) continue;
        const double SR = S - SL;
        const double score = SL * SL / (double)WL + SR * SR / (double)WR;
        if (!found || score > best) {
            float a = key_float(ws->key[i]), b = key_float(ws->key[i + 1]);
            float t = (float)((double)a + ((double)b - (double)a) * 0.5);
            if (!(t >= a && t < b)) t = a;
            best = score; bthr = t; found = 1;
        }
    }
    *out_score = best; *out_thr = bthr;
    return found;
}

static int64_t grow_reg(const reg_ctx *c, reg_ws *ws, dg_tree *t, int64_t lo, int64_t hi, int32_t depth) {
    int64_t id = tree_push(t);
    if (id < 0) return -1;
    if (depth > t->depth) t->depth = depth;
    const int32_t d = c->d;
    int64_t W = 0;
    double S = 0.0, ymin = 0.0, ymax = 0.0;
    for (int64_t i = lo; i < hi; ++i) {
        int32_t s = ws->samp[i];
        const double v = c->target[s];
        W += ws->w[s];
        S += (double)ws->w[s] * v;
        if (i == lo || v < ymin) ymin = v;
        if (i == lo || v > ymax) ymax = v;
    }
    t->card[id] = W;
    t->left[id] = -1; t->right[id] = -1; t->feature[id] = -1; t->threshold[id] = 0.0f; t->leaf_class[id] = 0;
    t->value[id] = (float)((c->eta > 0.0 ? c->eta : 1.0) * (S / (double)W));
    int32_t bf = -1;
    double bscore = 0.0;
    float bthr = 0.0f;
    if (ymin != ymax && W >= 2 * c->min_leaf && !(c->max_depth > 0 && depth >= c->max_depth)) {
        for (int32_t f = 0; f < d; ++f) ws->perm[f] = f;
        for (int32_t i = 0; i < d; ++i) {
            int32_t j = i + (int32_t)dg_bounded(&ws->rng, (uint64_t)(d - i));
            int32_t tmpf = ws->perm[i]; ws->perm[i] = ws->perm[j]; ws->perm[j] = tmpf;
            double score; float thr;
            if (best_split_reg(c, ws, lo, hi, ws->perm[i], S, W, &score, &thr)) {
                if (bf < 0 || score > bscore) { bf = ws->perm[i]; bscore = score; bthr = thr; }
            }
            if (i + 1 >= c->mtry && bf >= 0) break;
        }
    }
    if (bf < 0) {  /* a leaf: boosting adds its value to the rows that reach it */
        if (c->score)
            for (int64_t i = lo; i < hi; ++i) c->score[ws->samp[i]] += (double)t->value[id];
        return id;
    }
    int64_t nl = 0;
    for (int64_t i = lo; i < hi; ++i) {
        int32_t s = ws->samp[i];
        if (c->X[(int64_t)s * d + bf] <= bthr) ws->samp[lo + nl++] = s; else ws->tmp[i - lo - nl] = s;
    }
    memcpy(ws->samp + lo + nl, ws->tmp, sizeof(int32_t) * (size_t)(hi - lo - nl));
    t->feature[id] = bf;
    t->threshold[id] = bthr;
    t->leaf_class[id] = -1;
    t->value[id] = 0.0f;
    int64_t l = grow_reg(c, ws, t, lo, lo + nl, depth + 1);
    if (l < 0) return -1;
    int64_t r = grow_reg(c, ws, t, lo + nl, hi, depth + 1);
    if (r < 0) return -1;
    t->left[id] = (int32_t)l;
    t->right[id] = (int32_t)r;
    return id;
}

typedef struct { reg_ctx *c; int64_t next; pthread_mutex_t mu; int fail; } reg_pool;

static void *reg_forest_worker(void *arg) {
    reg_pool *p = (reg_pool *)arg;
    reg_ctx *c = p->c;
    reg_ws ws;
    int ok = reg_ws_alloc(&ws, c->n, c->d);
    for (;;) {
        pthread_mutex_lock(&p->mu);
        int64_t ti = p->next++;
        if (!ok) p->fail = 1;
        pthread_mutex_unlock(&p->mu);
        if (!ok || ti >= c->F->n_trees) break;
        dg_tree *t = &c->F->trees[ti];
        dg_rng_init(&ws.rng, c->seed, PURPOSE_TREE, (uint64_t)ti);
        memset(ws.w, 0, sizeof(int64_t) * (size_t)c->n);
        for (int64_t i = 0; i < c->n; ++i) ws.w[dg_bounded(&ws.rng, (uint64_t)c->n)]++;
        int64_t m = 0;
        for (int64_t i = 0; i < c->n; ++i)
            if (ws.w[i]) ws.samp[m++] = (int32_t)i;
        t->n_boot = c->n;
        if (grow_reg(c, &ws, t, 0, m, 0) < 0 || t->oom) {
            pthread_mutex_lock(&p->mu); p->fail = 1; pthread_mutex_unlock(&p->mu);
        }
    }
    reg_ws_free(&ws);
    return NULL;
}

/* Train a regression forest (eta == 0) or a boosted ensemble (eta > 0).
 * *base receives F_0 (boosting) or 0.  Returns NULL on bad arguments or
 * allocation failure. */
dg_forest *dg_train_regression(const float *X, const double *y, int64_t n, int32_t d, int32_t n_trees, int32_t mtry,
                               int32_t max_depth, int64_t min_leaf, double eta, uint64_t seed, double *base,
                               int n_threads) {
    if (n < 2 || n > INT32_MAX || d < 1 || n_trees < 1 || mtry < 1 || max_depth < 0 || min_leaf < 1 || eta < 0.0 ||
        !base)
        return NULL;
    dg_forest *F = calloc(1, sizeof(dg_forest));
    if (!F) return NULL;
    F->n_trees = n_trees; F->n_features = d; F->n_classes = 1;
    F->trees = calloc((size_t)n_trees, sizeof(dg_tree));
    if (!F->trees) { free(F); return NULL; }
    reg_ctx c = {X, y, n, d, mtry > d ? d : mtry, max_depth, min_leaf, seed, eta, F, y, NULL};
    *base = 0.0;
    if (eta == 0.0) {
        reg_pool p = {&c, 0, PTHREAD_MUTEX_INITIALIZER, 0};
        if (n_threads < 1) n_threads = 1;
        if (n_threads > n_trees) n_threads = n_trees;
        if (n_threads > 256) n_threads = 256;
        pthread_t th[256];
        for (int i = 0; i < n_threads; ++i) pthread_create(&th[i], NULL, reg_forest_worker, &p);
        for (int i = 0; i < n_threads; ++i) pthread_join(th[i], NULL);
        if (p.fail) { dg_forest_free(F); return NULL; }
        return F;
    }
    /* boosting: rounds are sequential */
    reg_ws ws;
    double *score = malloc(sizeof(double) * (size_t)n), *resid = malloc(sizeof(double) * (size_t)n);
    int ok = reg_ws_alloc(&ws, n, d) && score && resid;
    if (ok) {
        double s0 = 0.0;
        for (int64_t i = 0; i < n; ++i) s0 += y[i];
        *base = s0 / (double)n;
        for (int64_t i = 0; i < n; ++i) score[i] = *base;
        for (int64_t i = 0; i < n; ++i) ws.w[i] = 1;
        c.target = resid;
        c.score = score;
        for (int32_t m = 0; m < n_trees && ok; ++m) {
            for (int64_t i = 0; i < n; ++i) resid[i] = y[i] - score[i];
            for (int64_t i = 0; i < n; ++i) ws.samp[i] = (int32_t)i;
            dg_rng_init(&ws.rng, seed, PURPOSE_TREE, (uint64_t)m);
            dg_tree *t = &F->trees[m];
            t->n_boot = n;
            if (grow_reg(&c, &ws, t, 0, n, 0) < 0 || t->oom) ok = 0;
        }
    }
    reg_ws_free(&ws);
    free(score); free(resid);
    if (!ok) { dg_forest_free(F); return NULL; }
    return F;
}

/* Leaf values of every node (0 on internal nodes), in export order. */
void dg_forest_export_values(const dg_forest *F, float *value) {
    int64_t off = 0;
    for (int32_t t = 0; t < F->n_trees; ++t) {
        const dg_tree *tr = &F->trees[t];
        memcpy(value + off, tr->value, 4 * (size_t)tr->n_nodes);
        off += tr->n_nodes;
    }
}
