/*
 * dg_host.c - host build of the seeded input generator (dg_core.h), threaded
 * over rows.  Built with -ffp-contract=off so that its FP64 arithmetic is the
 * same sequence of correctly rounded operations as the device build.
 */
#include <pthread.h>
#include <stdlib.h>
#include <unistd.h>

#include "dg_core.h"

typedef struct {
    int kind; /* 0 random walk, 1 sinusoid */
    uint64_t seed;
    int64_t row0, begin, end;
    int n;
    float* out;
    const int64_t* idx; /* rows to generate (NULL: rows row0 + i) */
} dg_job;

static void* dg_worker(void* p) {
    dg_job* j = (dg_job*)p;
    double* buf = (double*)malloc(sizeof(double) * (size_t)j->n);
    if (!buf) return (void*)1;
    for (int64_t r = j->begin; r < j->end; ++r) {
        float* o = j->out + (size_t)(r - j->row0) * (size_t)j->n;
        const uint64_t row = j->idx ? (uint64_t)j->idx[r - j->row0] : (uint64_t)r;
        if (j->kind == 0)
            dg_random_walk_row(j->seed, row, j->n, buf, o);
        else
            dg_sinusoid_row(j->seed, row, j->n, buf, o);
    }
    free(buf);
    return NULL;
}

static int dg_run_idx(int kind, uint64_t seed, int64_t row0, int64_t count, int n, float* out,
                      int nthreads, const int64_t* idx);

static int dg_run(int kind, uint64_t seed, int64_t row0, int64_t count, int n, float* out,
                  int nthreads) {
    return dg_run_idx(kind, seed, row0, count, n, out, nthreads, NULL);
}

static int dg_run_idx(int kind, uint64_t seed, int64_t row0, int64_t count, int n, float* out,
                      int nthreads, const int64_t* idx) {
    if (n < 1 || n > DG_MAX_N || count < 0 || !out) return 1;
    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if ((int64_t)nthreads > count) nthreads = count > 0 ? (int)count : 1;
    pthread_t th[256];
    dg_job jobs[256];
    if (nthreads > 256) nthreads = 256;
    int rc = 0;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].kind = kind;
        jobs[t].seed = seed;
        jobs[t].row0 = row0;
        jobs[t].begin = row0 + count * t / nthreads;
        jobs[t].end = row0 + count * (t + 1) / nthreads;
        jobs[t].n = n;
        jobs[t].out = out;
        jobs[t].idx = idx;
    }
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[t], NULL, dg_worker, &jobs[t]) != 0) return 2;
    if (dg_worker(&jobs[0]) != NULL) rc = 3;
    for (int t = 1; t < nthreads; ++t) {
        void* r = NULL;
        pthread_join(th[t], &r);
        if (r != NULL) rc = 3;
    }
    return rc;
}

/* rows [row0, row0+count) of the z-normalised random-walk collection `seed` */
int dg_host_random_walks(uint64_t seed, int64_t row0, int64_t count, int n, float* out,
                         int nthreads) {
    return dg_run(0, seed, row0, count, n, out, nthreads);
}

/* rows [row0, row0+count) of the z-normalised sinusoid collection `seed` */
int dg_host_sinusoids(uint64_t seed, int64_t row0, int64_t count, int n, float* out,
                      int nthreads) {
    return dg_run(1, seed, row0, count, n, out, nthreads);
}

/* rows idx[0..count) (any order, repeats allowed) of collection (kind, seed) */
int dg_host_rows_at(int kind, uint64_t seed, const int64_t* idx, int64_t count, int n, float* out,
                    int nthreads) {
    return dg_run_idx(kind, seed, 0, count, n, out, nthreads, idx);
}

/* noisy copies: out[b] = znorm(members[b] + sigma[b] * N(0,1)), noise stream
 * (qseed, qid0 + b) */
int dg_host_noisy(const float* members, uint64_t qseed, int64_t qid0, int64_t count, int n,
                  const double* sigma, float* out) {
    if (n < 1 || n > DG_MAX_N) return 1;
    double* buf = (double*)malloc(sizeof(double) * (size_t)n);
    if (!buf) return 2;
    for (int64_t b = 0; b < count; ++b)
        dg_noisy_row(members + (size_t)b * n, qseed, (uint64_t)(qid0 + b), n, sigma[b], buf,
                     out + (size_t)b * n);
    free(buf);
    return 0;
}

/* member index in [0, N) for queries qid0 .. qid0+count-1 */
void dg_host_pick_members(uint64_t qseed, int64_t qid0, int64_t count, uint64_t N,
                          int64_t* out) {
    for (int64_t b = 0; b < count; ++b)
        out[b] = (int64_t)dg_pick_member(qseed, (uint64_t)(qid0 + b), N);
}

/* test hooks for the building blocks */
void dg_host_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    dg_u32x4 c;
    for (int i = 0; i < 4; ++i) c.v[i] = ctr[i];
    dg_u32x4 r = dg_philox4x32_10(c, key[0], key[1]);
    for (int i = 0; i < 4; ++i) out[i] = r.v[i];
}
double dg_host_ln(double x) { return dg_ln(x); }
void dg_host_sincos_turns(double u, double* s, double* c) { dg_sincos_turns(u, s, c); }
void dg_host_normal_pair(uint64_t seed, uint64_t row, uint32_t d, uint32_t tag, double* z0,
                         double* z1) {
    dg_normal_pair(seed, row, d, tag, z0, z1);
}
