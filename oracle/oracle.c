/*
 * oracle.c - CPU oracle for exact Euclidean k-NN over data series with an
 * iSAX index.  TEST INFRASTRUCTURE ONLY: it is called by the tests, by the
 * smoke check and by the benchmark's CPU-baseline leg, never by the GPU
 * library.  It shares no code with the GPU path.
 *
 * Everything is plain FP64, single pass, written to be checked against the
 * paper by eye (compile with -ffp-contract=off so no multiply-add is fused):
 *
 *   or_breakpoints   beta_t = Phi^{-1}(t / card), t = 1..card-1: the
 *                    equiprobable N(0,1) region boundaries that split the
 *                    y-axis into the iSAX symbol regions (Section II, iSAX
 *                    Representation), found by bisection on Phi(x) =
 *                    erfc(-x / sqrt 2) / 2.
 *   or_paa           segment means of w equal-length segments (Section II,
 *                    PAA).
 *   or_symbol        symbol = number of breakpoints <= value, so a value on a
 *                    breakpoint belongs to the upper region.
 *   or_ed2           squared Euclidean distance sum_j (x_j - q_j)^2, summed
 *                    left to right (Section II, Similarity Search).
 *   or_lb2_*         iSAX lower bound: (n/w) sum_i dist(qpaa_i, region_i)^2,
 *                    the distance from the query's PAA value to the region a
 *                    series' (or a node's) symbol covers (Section III: pruning
 *                    of series and of subtrees with lower-bound distances).
 *   or_bruteforce    the definition of the answer: all N distances, the k
 *                    smallest by (distance, index) (Section II, Similarity
 *                    Search; k > 1 generalises 1-NN).
 *   or_index_*       an ADS+-style tree (Section II, ADS+ Index): root with up
 *                    to 2^w children keyed by the first bit of every segment,
 *                    binary inner nodes, leaves that split when they exceed
 *                    their capacity on the segment whose extra bit gives the
 *                    most balanced split; and MESSI's exact search (Section
 *                    III, MESSI Approach): approximate answer from the leaf the
 *                    query descends to, subtree pruning against the BSF, leaves
 *                    processed in lower-bound order from a priority queue,
 *                    series lower bound, then real distance, BSF updates, stop
 *                    at the first leaf whose bound exceeds the BSF.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define OR_W_MAX 16

/* ------------------------------------------------------------ breakpoints */
static double or_phi(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* beta[t-1] = Phi^{-1}(t / card).  Lower half (p < 1/2) by bisection on Phi,
 * where erfc of a positive argument is accurate to a few ulps relative; the
 * middle one is 0 and the upper half follows from Phi^{-1}(1 - p) =
 * -Phi^{-1}(p), so the table is exactly antisymmetric. */
void or_breakpoints(int card, double* beta) {
    for (int t = 1; 2 * t < card; ++t) {
        double p = (double)t / (double)card;
        double lo = -40.0, hi = 0.0; /* Phi(lo) < p <= Phi(hi) */
        for (int it = 0; it < 5000; ++it) {
            double mid = lo + (hi - lo) / 2.0;
            if (mid == lo || mid == hi) break;
            if (or_phi(mid) < p)
                lo = mid;
            else
                hi = mid;
        }
        beta[t - 1] = (fabs(or_phi(lo) - p) < fabs(or_phi(hi) - p)) ? lo : hi;
        beta[card - t - 1] = -beta[t - 1];
    }
    beta[card / 2 - 1] = 0.0;
}

/* ------------------------------------------------------------ PAA, SAX */
void or_paa(const float* x, int n, int w, double* paa) {
    int m = n / w;
    for (int i = 0; i < w; ++i) {
        double s = 0.0;
        for (int j = 0; j < m; ++j) s += (double)x[i * m + j];
        paa[i] = s / (double)m;
    }
}

int or_symbol(double v, const double* beta, int card) {
    int s = 0;
    for (int t = 0; t < card - 1; ++t)
        if (beta[t] <= v) s++;
    return s;
}

/* PAA and symbols of N series */
void or_summarize(const float* X, int64_t N, int n, int w, int card, const double* beta,
                  double* paa_out, uint8_t* sax_out) {
    double paa[OR_W_MAX];
    for (int64_t r = 0; r < N; ++r) {
        or_paa(X + (size_t)r * n, n, w, paa);
        for (int i = 0; i < w; ++i) {
            if (paa_out) paa_out[(size_t)r * w + i] = paa[i];
            if (sax_out) sax_out[(size_t)r * w + i] = (uint8_t)or_symbol(paa[i], beta, card);
        }
    }
}

/* ------------------------------------------------------------ distances */
double or_ed2(const float* x, const float* q, int n) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
        double d = (double)x[j] - (double)q[j];
        s += d * d;
    }
    return s;
}

/* lower edge of symbol region s (beta_0 = -inf) and upper edge (beta_card = +inf) */
static double or_edge(const double* beta, int card, int t) {
    if (t <= 0) return -INFINITY;
    if (t >= card) return INFINITY;
    return beta[t - 1];
}

static double or_region_dist(double v, double lo, double hi) {
    if (v < lo) return lo - v;
    if (v > hi) return v - hi;
    return 0.0;
}

/* lower bound (squared) of a series with full-cardinality symbols */
double or_lb2_series(const double* qpaa, const uint8_t* sym, int w, int n, const double* beta,
                     int card) {
    double s = 0.0;
    for (int i = 0; i < w; ++i) {
        double d = or_region_dist(qpaa[i], or_edge(beta, card, sym[i]),
                                  or_edge(beta, card, sym[i] + 1));
        s += d * d;
    }
    return (double)(n / w) * s;
}

/* lower bound (squared) of a node: per segment a prefix value `val` of
 * `bits` bits out of cbits, i.e. the symbol range [val << (cbits-bits),
 * ((val+1) << (cbits-bits)) - 1] */
double or_lb2_node(const double* qpaa, const uint16_t* val, const uint8_t* bits, int w, int n,
                   const double* beta, int card, int cbits) {
    double s = 0.0;
    for (int i = 0; i < w; ++i) {
        int sh = cbits - bits[i];
        int lo = (int)val[i] << sh;
        int hi = (((int)val[i] + 1) << sh) - 1;
        double d = or_region_dist(qpaa[i], or_edge(beta, card, lo), or_edge(beta, card, hi + 1));
        s += d * d;
    }
    return (double)(n / w) * s;
}

/* ------------------------------------------------------------ top-k list */
typedef struct {
    int k, cnt;
    double* d;
    int64_t* id;
} or_topk;

static int or_less(double d1, int64_t i1, double d2, int64_t i2) {
    return d1 < d2 || (d1 == d2 && i1 < i2);
}

static void or_topk_push(or_topk* t, double d, int64_t id) {
    if (t->cnt == t->k && !or_less(d, id, t->d[t->k - 1], t->id[t->k - 1])) return;
    int p = t->cnt < t->k ? t->cnt : t->k - 1;
    while (p > 0 && or_less(d, id, t->d[p - 1], t->id[p - 1])) {
        t->d[p] = t->d[p - 1];
        t->id[p] = t->id[p - 1];
        --p;
    }
    t->d[p] = d;
    t->id[p] = id;
    if (t->cnt < t->k) t->cnt++;
}

static double or_topk_thr(const or_topk* t) { return t->cnt < t->k ? INFINITY : t->d[t->k - 1]; }

/* ------------------------------------------------------------ brute force */
typedef struct {
    const float* X;
    const float* Q;
    int64_t r0, r1;
    int n, B, k;
    double* d;     /* [B][k] */
    int64_t* id;   /* [B][k] */
    int* cnt;      /* [B] */
} or_bf_job;

static void* or_bf_worker(void* p) {
    or_bf_job* j = (or_bf_job*)p;
    /* rows in blocks of 512 so a block stays in cache across the queries */
    for (int64_t r0 = j->r0; r0 < j->r1; r0 += 512) {
        int64_t r1 = r0 + 512 < j->r1 ? r0 + 512 : j->r1;
        for (int b = 0; b < j->B; ++b) {
            or_topk t = {j->k, j->cnt[b], j->d + (size_t)b * j->k, j->id + (size_t)b * j->k};
            const float* q = j->Q + (size_t)b * j->n;
            for (int64_t r = r0; r < r1; ++r) or_topk_push(&t, or_ed2(j->X + (size_t)r * j->n, q, j->n), r);
            j->cnt[b] = t.cnt;
        }
    }
    return NULL;
}

/* exact k-NN of B queries by scanning all N rows: out_id/out_d2 [B][k],
 * ascending by (squared distance, row index).  Threads split the rows; their
 * partial lists are merged with the same ordering. */
int or_bruteforce(const float* X, int64_t N, int n, const float* Q, int B, int k, int nthreads,
                  int64_t* out_id, double* out_d2) {
    if (k < 1 || N < 1) return 1;
    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > N) nthreads = (int)N;
    or_bf_job* jobs = (or_bf_job*)calloc((size_t)nthreads, sizeof(or_bf_job));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    double* d = (double*)malloc(sizeof(double) * (size_t)nthreads * B * k);
    int64_t* id = (int64_t*)malloc(sizeof(int64_t) * (size_t)nthreads * B * k);
    int* cnt = (int*)calloc((size_t)nthreads * B, sizeof(int));
    if (!jobs || !th || !d || !id || !cnt) return 2;
    for (int t = 0; t < nthreads; ++t) {
        or_bf_job j = {X, Q, N * t / nthreads, N * (t + 1) / nthreads, n, B, k,
                       d + (size_t)t * B * k, id + (size_t)t * B * k, cnt + (size_t)t * B};
        jobs[t] = j;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, or_bf_worker, &jobs[t]);
    or_bf_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    for (int b = 0; b < B; ++b) {
        or_topk tk = {k, 0, out_d2 + (size_t)b * k, out_id + (size_t)b * k};
        for (int t = 0; t < nthreads; ++t) {
            const or_bf_job* j = &jobs[t];
            for (int i = 0; i < j->cnt[b]; ++i)
                or_topk_push(&tk, j->d[(size_t)b * k + i], j->id[(size_t)b * k + i]);
        }
        for (int i = tk.cnt; i < k; ++i) {
            out_d2[(size_t)b * k + i] = INFINITY;
            out_id[(size_t)b * k + i] = -1;
        }
    }
    free(jobs);
    free(th);
    free(d);
    free(id);
    free(cnt);
    return 0;
}

/* ------------------------------------------------------------ iSAX index */
typedef struct or_node {
    int leaf;
    int split_seg;
    uint8_t bits[OR_W_MAX];
    uint16_t val[OR_W_MAX];
    struct or_node* child[2];
    int64_t* ids;
    int64_t cnt, cap;
} or_node;

typedef struct {
    int64_t N;
    int n, w, card, cbits, leaf_cap;
    const float* X; /* borrowed: must outlive the index */
    double* beta;
    uint8_t* sax;
    or_node** root;
    double maxabs;
    int64_t nodes, leaves;
} or_index;

typedef struct {
    int64_t leaves_total, leaves_queued, leaves_visited, series_lb, series_ed;
} or_stats;

static or_node* or_new_leaf(void) {
    or_node* nd = (or_node*)calloc(1, sizeof(or_node));
    if (!nd) return NULL;
    nd->leaf = 1;
    nd->split_seg = -1;
    return nd;
}

static void or_leaf_append(or_node* nd, int64_t id) {
    if (nd->cnt == nd->cap) {
        nd->cap = nd->cap ? nd->cap * 2 : 16;
        nd->ids = (int64_t*)realloc(nd->ids, sizeof(int64_t) * (size_t)nd->cap);
    }
    nd->ids[nd->cnt++] = id;
}

/* bit of symbol s that a child of a node with `b` bits on that segment adds */
static int or_next_bit(int s, int b, int cbits) { return (s >> (cbits - b - 1)) & 1; }

static void or_split(or_index* ix, or_node* nd) {
    int best = -1;
    int64_t best_bal = 0;
    for (int g = 0; g < ix->w; ++g) {
        if (nd->bits[g] >= ix->cbits) continue;
        int64_t ones = 0;
        for (int64_t i = 0; i < nd->cnt; ++i)
            ones += or_next_bit(ix->sax[(size_t)nd->ids[i] * ix->w + g], nd->bits[g], ix->cbits);
        int64_t bal = llabs(2 * ones - nd->cnt);
        if (best < 0 || bal < best_bal) {
            best = g;
            best_bal = bal;
        }
    }
    if (best < 0) return; /* every segment at full cardinality: leaf stays over capacity */
    for (int c = 0; c < 2; ++c) {
        or_node* ch = or_new_leaf();
        memcpy(ch->bits, nd->bits, sizeof nd->bits);
        memcpy(ch->val, nd->val, sizeof nd->val);
        ch->bits[best] = (uint8_t)(nd->bits[best] + 1);
        ch->val[best] = (uint16_t)(nd->val[best] * 2 + c);
        nd->child[c] = ch;
    }
    for (int64_t i = 0; i < nd->cnt; ++i) {
        int64_t id = nd->ids[i];
        int b = or_next_bit(ix->sax[(size_t)id * ix->w + best], nd->bits[best], ix->cbits);
        or_leaf_append(nd->child[b], id);
    }
    free(nd->ids);
    nd->ids = NULL;
    nd->cnt = nd->cap = 0;
    nd->leaf = 0;
    nd->split_seg = best;
    ix->nodes += 2;
    ix->leaves += 1;
    for (int c = 0; c < 2; ++c)
        if (nd->child[c]->cnt > ix->leaf_cap) or_split(ix, nd->child[c]);
}

static int or_root_key(const uint8_t* sym, int w, int cbits) {
    int key = 0;
    for (int i = 0; i < w; ++i) key = (key << 1) | ((sym[i] >> (cbits - 1)) & 1);
    return key;
}

static void or_insert(or_index* ix, int64_t id) {
    const uint8_t* sym = ix->sax + (size_t)id * ix->w;
    int key = or_root_key(sym, ix->w, ix->cbits);
    or_node* nd = ix->root[key];
    if (!nd) {
        nd = or_new_leaf();
        for (int i = 0; i < ix->w; ++i) {
            nd->bits[i] = 1;
            nd->val[i] = (uint16_t)((sym[i] >> (ix->cbits - 1)) & 1);
        }
        ix->root[key] = nd;
        ix->nodes++;
        ix->leaves++;
    }
    while (!nd->leaf) {
        int g = nd->split_seg;
        nd = nd->child[or_next_bit(sym[g], nd->bits[g], ix->cbits)];
    }
    or_leaf_append(nd, id);
    if (nd->cnt > ix->leaf_cap) or_split(ix, nd);
}

void* or_index_build(const float* X, int64_t N, int n, int w, int card, int leaf_cap) {
    if (N < 1 || w < 1 || w > OR_W_MAX || n % w || card < 2 || card > 256 || (card & (card - 1)) ||
        leaf_cap < 1)
        return NULL;
    or_index* ix = (or_index*)calloc(1, sizeof(or_index));
    ix->N = N;
    ix->n = n;
    ix->w = w;
    ix->card = card;
    ix->cbits = 0;
    while ((1 << ix->cbits) < card) ix->cbits++;
    ix->leaf_cap = leaf_cap;
    ix->X = X;
    ix->beta = (double*)malloc(sizeof(double) * (size_t)card);
    or_breakpoints(card, ix->beta);
    ix->sax = (uint8_t*)malloc((size_t)N * w);
    or_summarize(X, N, n, w, card, ix->beta, NULL, ix->sax);
    ix->root = (or_node**)calloc((size_t)1 << w, sizeof(or_node*));
    double mx = 0.0;
    for (int64_t i = 0; i < N * n; ++i) {
        double a = fabs((double)X[i]);
        if (a > mx) mx = a;
    }
    ix->maxabs = mx;
    for (int64_t i = 0; i < N; ++i) or_insert(ix, i);
    return ix;
}

static void or_free_node(or_node* nd) {
    if (!nd) return;
    or_free_node(nd->child[0]);
    or_free_node(nd->child[1]);
    free(nd->ids);
    free(nd);
}

void or_index_free(void* p) {
    or_index* ix = (or_index*)p;
    if (!ix) return;
    for (int64_t k = 0; k < ((int64_t)1 << ix->w); ++k) or_free_node(ix->root[k]);
    free(ix->root);
    free(ix->sax);
    free(ix->beta);
    free(ix);
}

int64_t or_index_leaves(const void* p) { return ((const or_index*)p)->leaves; }

/* leaf sizes in depth-first order (root children by key, child 0 first) */
static void or_collect(const or_node* nd, int64_t* out, int64_t* pos) {
    if (!nd) return;
    if (nd->leaf) {
        if (out) out[*pos] = nd->cnt;
        (*pos)++;
        return;
    }
    or_collect(nd->child[0], out, pos);
    or_collect(nd->child[1], out, pos);
}

int64_t or_index_leaf_sizes(const void* p, int64_t* out) {
    const or_index* ix = (const or_index*)p;
    int64_t pos = 0;
    for (int64_t k = 0; k < ((int64_t)1 << ix->w); ++k) or_collect(ix->root[k], out, &pos);
    return pos;
}

/* member ids of every leaf, leaf after leaf in the depth-first order above,
 * each leaf's ids in insertion (row) order; returns N */
static void or_collect_ids(const or_node* nd, int64_t* out, int64_t* pos) {
    if (!nd) return;
    if (nd->leaf) {
        for (int64_t i = 0; i < nd->cnt; ++i) out[(*pos)++] = nd->ids[i];
        return;
    }
    or_collect_ids(nd->child[0], out, pos);
    or_collect_ids(nd->child[1], out, pos);
}

int64_t or_index_leaf_ids(const void* p, int64_t* out) {
    const or_index* ix = (const or_index*)p;
    int64_t pos = 0;
    for (int64_t k = 0; k < ((int64_t)1 << ix->w); ++k) or_collect_ids(ix->root[k], out, &pos);
    return pos;
}

/* ---- priority queue of (lower bound, leaf) ordered by bound, then insertion */
typedef struct {
    double lb;
    int64_t seq;
    const or_node* nd;
} or_pq_item;

typedef struct {
    or_pq_item* a;
    int64_t n, cap;
} or_pq;

static int or_pq_less(const or_pq_item* x, const or_pq_item* y) {
    return x->lb < y->lb || (x->lb == y->lb && x->seq < y->seq);
}

static void or_pq_push(or_pq* q, or_pq_item it) {
    if (q->n == q->cap) {
        q->cap = q->cap ? q->cap * 2 : 64;
        q->a = (or_pq_item*)realloc(q->a, sizeof(or_pq_item) * (size_t)q->cap);
    }
    int64_t i = q->n++;
    q->a[i] = it;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!or_pq_less(&q->a[i], &q->a[p])) break;
        or_pq_item t = q->a[i];
        q->a[i] = q->a[p];
        q->a[p] = t;
        i = p;
    }
}

static or_pq_item or_pq_pop(or_pq* q) {
    or_pq_item top = q->a[0];
    q->a[0] = q->a[--q->n];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < q->n && or_pq_less(&q->a[l], &q->a[m])) m = l;
        if (r < q->n && or_pq_less(&q->a[r], &q->a[m])) m = r;
        if (m == i) break;
        or_pq_item t = q->a[i];
        q->a[i] = q->a[m];
        q->a[m] = t;
        i = m;
    }
    return top;
}

typedef struct {
    const or_index* ix;
    const float* q;
    double qpaa[OR_W_MAX];
    double slack_abs; /* absolute slack on the lower bound distance (not squared) */
    or_topk top;
    or_pq pq;
    int64_t seq;
    const or_node* approx;
    or_stats* st;
} or_search;

/* a bound proves a candidate worse than the current k-th best only if it
 * exceeds it by more than the FP64 rounding of PAA, bound and distance */
static int or_prunes(const or_search* s, double lb2) {
    double thr = or_topk_thr(&s->top);
    if (isinf(thr)) return 0;
    return sqrt(lb2) > sqrt(thr) * (1.0 + 1e-10) + s->slack_abs;
}

static void or_scan_leaf(or_search* s, const or_node* nd) {
    const or_index* ix = s->ix;
    for (int64_t i = 0; i < nd->cnt; ++i) {
        int64_t id = nd->ids[i];
        double lb2 = or_lb2_series(s->qpaa, ix->sax + (size_t)id * ix->w, ix->w, ix->n, ix->beta,
                                   ix->card);
        if (s->st) s->st->series_lb++;
        if (or_prunes(s, lb2)) continue;
        if (s->st) s->st->series_ed++;
        or_topk_push(&s->top, or_ed2(ix->X + (size_t)id * ix->n, s->q, ix->n), id);
    }
}

static void or_traverse(or_search* s, const or_node* nd) {
    const or_index* ix = s->ix;
    double lb2 = or_lb2_node(s->qpaa, nd->val, nd->bits, ix->w, ix->n, ix->beta, ix->card, ix->cbits);
    if (or_prunes(s, lb2)) return;
    if (nd->leaf) {
        if (nd != s->approx && nd->cnt > 0) {
            or_pq_item it = {lb2, s->seq++, nd};
            or_pq_push(&s->pq, it);
            if (s->st) s->st->leaves_queued++;
        }
        return;
    }
    or_traverse(s, nd->child[0]);
    or_traverse(s, nd->child[1]);
}

/* exact k-NN of one query; out_id/out_d2 [k] ascending by (squared distance, index) */
int or_index_query(const void* p, const float* q, int k, int64_t* out_id, double* out_d2,
                   or_stats* st) {
    const or_index* ix = (const or_index*)p;
    if (k < 1) return 1;
    or_search s;
    memset(&s, 0, sizeof s);
    s.ix = ix;
    s.q = q;
    s.st = st;
    if (st) memset(st, 0, sizeof *st);
    if (st) st->leaves_total = ix->leaves;
    s.top.k = k;
    s.top.d = out_d2;
    s.top.id = out_id;
    or_paa(q, ix->n, ix->w, s.qpaa);
    double qmax = 0.0;
    for (int j = 0; j < ix->n; ++j)
        if (fabs((double)q[j]) > qmax) qmax = fabs((double)q[j]);
    int m = ix->n / ix->w;
    s.slack_abs = sqrt((double)ix->n) * (double)(m + 2) * ldexp(1.0, -52) * (ix->maxabs + qmax);

    /* approximate answer: the leaf the query's own iSAX word descends to */
    uint8_t qsym[OR_W_MAX];
    for (int i = 0; i < ix->w; ++i) qsym[i] = (uint8_t)or_symbol(s.qpaa[i], ix->beta, ix->card);
    int key = or_root_key(qsym, ix->w, ix->cbits);
    const or_node* nd = ix->root[key];
    if (!nd) { /* no such root child: take the child with the smallest bound */
        double best = INFINITY;
        for (int64_t c = 0; c < ((int64_t)1 << ix->w); ++c) {
            const or_node* r = ix->root[c];
            if (!r) continue;
            double lb2 = or_lb2_node(s.qpaa, r->val, r->bits, ix->w, ix->n, ix->beta, ix->card,
                                     ix->cbits);
            if (lb2 < best) {
                best = lb2;
                nd = r;
            }
        }
    }
    while (nd && !nd->leaf) {
        int g = nd->split_seg;
        nd = nd->child[or_next_bit(qsym[g], nd->bits[g], ix->cbits)];
    }
    s.approx = nd;
    if (nd) {
        or_scan_leaf(&s, nd);
        if (st) st->leaves_visited++;
    }

    /* exact answer: prune subtrees, queue leaves by bound, pop in order */
    for (int64_t c = 0; c < ((int64_t)1 << ix->w); ++c)
        if (ix->root[c]) or_traverse(&s, ix->root[c]);
    while (s.pq.n > 0) {
        or_pq_item it = or_pq_pop(&s.pq);
        if (or_prunes(&s, it.lb)) break;
        if (st) st->leaves_visited++;
        or_scan_leaf(&s, it.nd);
    }
    free(s.pq.a);
    for (int i = s.top.cnt; i < k; ++i) {
        out_d2[i] = INFINITY;
        out_id[i] = -1;
    }
    return 0;
}
