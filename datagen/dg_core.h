/*
 * dg_core.h - seeded synthetic input generator shared by the CPU oracle and
 * the GPU path (the only code the two sides share).  It holds none of the
 * indexing method's arithmetic: it only produces the collections and queries
 * the method is run on.
 *
 * Every value is a pure function of (seed, row, draw index), so any row can be
 * regenerated on its own, on the host or on the device, with identical bits:
 *
 *   - random bits:  Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 *     numbers: as easy as 1, 2, 3", SC'11), counter = (row lo, row hi, draw,
 *     stream tag), key = (seed lo, seed hi);
 *   - uniforms:     53-bit doubles k * 2^-53 built from two 32-bit outputs;
 *   - normals:      Box-Muller transform (Box & Muller 1958) in FP64;
 *   - ln and sin/cos used by Box-Muller are written here from their series
 *     (atanh series for ln, Taylor series after exact octant reduction for
 *     sin/cos) using only +, -, *, / and sqrt with round-to-nearest and no
 *     fused multiply-add, so the host (built with -ffp-contract=off) and the
 *     device (explicit __d*_rn intrinsics) evaluate the same IEEE operations.
 *
 * Workloads (all rows z-normalised: population mean 0, population std 1,
 * computed in FP64, then rounded to fp32):
 *   - random walk:  x_j = sum_{t<=j} z_t, z_t ~ N(0,1)             (the paper's
 *                   "Synthetic" dataset shape, Section IV)
 *   - sinusoids:    x_t = sum_{c=1..3} a_c sin(2 pi (f_c t / n + u_c))
 *                         + 0.3 z_t, f ~ U[1,20), u ~ U[0,1), a ~ U[0.5,2)
 *   - noisy member: member row + sigma * z_t, re-z-normalised.
 */
#ifndef ISAX_DG_CORE_H
#define ISAX_DG_CORE_H

#include <stdint.h>

#if defined(__CUDACC__)
#define DG_FN __host__ __device__ static inline
#else
#define DG_FN static inline
#endif

#if defined(__CUDA_ARCH__)
#define DG_ADD(a, b) __dadd_rn((a), (b))
#define DG_SUB(a, b) __dsub_rn((a), (b))
#define DG_MUL(a, b) __dmul_rn((a), (b))
#define DG_DIV(a, b) __ddiv_rn((a), (b))
#define DG_SQRT(a) __dsqrt_rn(a)
#define DG_TOF32(a) __double2float_rn(a)
#else
#include <math.h>
#include <string.h>
#define DG_ADD(a, b) ((a) + (b))
#define DG_SUB(a, b) ((a) - (b))
#define DG_MUL(a, b) ((a) * (b))
#define DG_DIV(a, b) ((a) / (b))
#define DG_SQRT(a) sqrt(a)
#define DG_TOF32(a) ((float)(a))
#endif

#define DG_MAX_N 4096

/* stream tags (fourth counter word) */
#define DG_TAG_STEPS 0u   /* N(0,1) steps / noise of a data row */
#define DG_TAG_PARAMS 1u  /* sinusoid parameters of a data row */
#define DG_TAG_QNOISE 2u  /* noise added to a member query */
#define DG_TAG_QPICK 3u   /* which member a query copies */

/* ---------------------------------------------------------------- Philox */
typedef struct { uint32_t v[4]; } dg_u32x4;

DG_FN void dg_mulhilo(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

/* Philox4x32 with 10 rounds: multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key
 * increments 0x9E3779B9 / 0xBB67AE85, as published. */
DG_FN dg_u32x4 dg_philox4x32_10(dg_u32x4 c, uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        dg_mulhilo(0xD2511F53u, c.v[0], &hi0, &lo0);
        dg_mulhilo(0xCD9E8D57u, c.v[2], &hi1, &lo1);
        dg_u32x4 n;
        n.v[0] = hi1 ^ c.v[1] ^ k0;
        n.v[1] = lo1;
        n.v[2] = hi0 ^ c.v[3] ^ k1;
        n.v[3] = lo0;
        c = n;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

DG_FN dg_u32x4 dg_draw(uint64_t seed, uint64_t row, uint32_t draw, uint32_t tag) {
    dg_u32x4 c;
    c.v[0] = (uint32_t)row;
    c.v[1] = (uint32_t)(row >> 32);
    c.v[2] = draw;
    c.v[3] = tag;
    return dg_philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
}

/* k * 2^-53 in [0, 1 - 2^-53] from two 32-bit words (exact) */
DG_FN double dg_u53(uint32_t a, uint32_t b) {
    uint64_t k = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
    return (double)k * 0x1.0p-53;
}

/* ---------------------------------------------------------------- ln, sincos */
DG_FN uint64_t dg_dbits(double x) {
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    memcpy(&b, &x, sizeof b);
    return b;
#endif
}
DG_FN double dg_bitsd(uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double x;
    memcpy(&x, &b, sizeof x);
    return x;
#endif
}

/* natural log of a positive normal double: x = 2^e f, f in [sqrt(2)/2, sqrt(2)],
 * ln f = 2 atanh(s), s = (f-1)/(f+1), |s| <= 0.1716, series to s^27. */
DG_FN double dg_ln(double x) {
    uint64_t b = dg_dbits(x);
    int e = (int)((b >> 52) & 0x7ff) - 1023;
    double f = dg_bitsd((b & 0x000fffffffffffffull) | 0x3ff0000000000000ull);
    if (f > 0x1.6a09e667f3bcdp+0) {
        f = DG_MUL(f, 0.5);
        e += 1;
    }
    double s = DG_DIV(DG_SUB(f, 1.0), DG_ADD(f, 1.0));
    double z = DG_MUL(s, s);
    double p = 0x1.2f684bda12f68p-5; /* 1/27 */
    p = DG_ADD(DG_MUL(p, z), 0x1.47ae147ae147bp-5); /* 1/25 */
    p = DG_ADD(DG_MUL(p, z), 0x1.642c8590b2164p-5); /* 1/23 */
    p = DG_ADD(DG_MUL(p, z), 0x1.8618618618618p-5); /* 1/21 */
    p = DG_ADD(DG_MUL(p, z), 0x1.af286bca1af28p-5); /* 1/19 */
    p = DG_ADD(DG_MUL(p, z), 0x1.e1e1e1e1e1e1ep-5); /* 1/17 */
    p = DG_ADD(DG_MUL(p, z), 0x1.1111111111111p-4); /* 1/15 */
    p = DG_ADD(DG_MUL(p, z), 0x1.3b13b13b13b14p-4); /* 1/13 */
    p = DG_ADD(DG_MUL(p, z), 0x1.745d1745d1746p-4); /* 1/11 */
    p = DG_ADD(DG_MUL(p, z), 0x1.c71c71c71c71cp-4); /* 1/9 */
    p = DG_ADD(DG_MUL(p, z), 0x1.2492492492492p-3); /* 1/7 */
    p = DG_ADD(DG_MUL(p, z), 0x1.999999999999ap-3); /* 1/5 */
    p = DG_ADD(DG_MUL(p, z), 0x1.5555555555555p-2); /* 1/3 */
    p = DG_ADD(DG_MUL(p, z), 1.0);
    double lnf = DG_MUL(DG_MUL(2.0, s), p);
    double de = (double)e;
    /* ln 2 split so that e * hi is exact for |e| < 2^20 */
    return DG_ADD(DG_MUL(de, 0x1.62e42fee00000p-1),
                  DG_ADD(DG_MUL(de, 0x1.a39ef35793c76p-33), lnf));
}

/* sin and cos of a in [0, pi/4] by Taylor series (truncation < 1e-19) */
DG_FN void dg_sincos_small(double a, double* sn, double* cs) {
    double z = DG_MUL(a, a);
    double ps = -0x1.2f49b46814157p-57; /* -1/19! */
    ps = DG_ADD(DG_MUL(ps, z), 0x1.952c77030ad4ap-49);  /* 1/17! */
    ps = DG_ADD(DG_MUL(ps, z), -0x1.ae7f3e733b81fp-41); /* -1/15! */
    ps = DG_ADD(DG_MUL(ps, z), 0x1.6124613a86d09p-33);  /* 1/13! */
    ps = DG_ADD(DG_MUL(ps, z), -0x1.ae64567f544e4p-26); /* -1/11! */
    ps = DG_ADD(DG_MUL(ps, z), 0x1.71de3a556c734p-19);  /* 1/9! */
    ps = DG_ADD(DG_MUL(ps, z), -0x1.a01a01a01a01ap-13); /* -1/7! */
    ps = DG_ADD(DG_MUL(ps, z), 0x1.1111111111111p-7);   /* 1/5! */
    ps = DG_ADD(DG_MUL(ps, z), -0x1.5555555555555p-3);  /* -1/3! */
    *sn = DG_ADD(a, DG_MUL(DG_MUL(a, z), ps));
    double pc = 0x1.e542ba4020225p-62; /* 1/20! */
    pc = DG_ADD(DG_MUL(pc, z), -0x1.6827863b97d97p-53); /* -1/18! */
    pc = DG_ADD(DG_MUL(pc, z), 0x1.ae7f3e733b81fp-45);  /* 1/16! */
    pc = DG_ADD(DG_MUL(pc, z), -0x1.93974a8c07c9dp-37); /* -1/14! */
    pc = DG_ADD(DG_MUL(pc, z), 0x1.1eed8eff8d898p-29);  /* 1/12! */
    pc = DG_ADD(DG_MUL(pc, z), -0x1.27e4fb7789f5cp-22); /* -1/10! */
    pc = DG_ADD(DG_MUL(pc, z), 0x1.a01a01a01a01ap-16);  /* 1/8! */
    pc = DG_ADD(DG_MUL(pc, z), -0x1.6c16c16c16c17p-10); /* -1/6! */
    pc = DG_ADD(DG_MUL(pc, z), 0x1.5555555555555p-5);   /* 1/4! */
    pc = DG_ADD(DG_MUL(pc, z), -0.5);                   /* -1/2! */
    *cs = DG_ADD(1.0, DG_MUL(z, pc));
}

/* sin and cos of 2*pi*u for u in [0, 1): exact octant reduction (8u, its
 * integer part and the complement 1 - f are exact for the inputs used here),
 * then the small-angle series and the octant symmetries. */
DG_FN void dg_sincos_turns(double u, double* sn, double* cs) {
    double t = DG_MUL(u, 8.0);
    int o = (int)t;
    if (o > 7) o = 7;
    if (o < 0) o = 0;
    double f = DG_SUB(t, (double)o);
    double r = (o & 1) ? DG_SUB(1.0, f) : f;
    double s, c;
    dg_sincos_small(DG_MUL(r, 0x1.921fb54442d18p-1), &s, &c);
    switch (o) {
        case 0: *sn = s;  *cs = c;  break;
        case 1: *sn = c;  *cs = s;  break;
        case 2: *sn = c;  *cs = -s; break;
        case 3: *sn = s;  *cs = -c; break;
        case 4: *sn = -s; *cs = -c; break;
        case 5: *sn = -c; *cs = -s; break;
        case 6: *sn = -c; *cs = s;  break;
        default: *sn = -s; *cs = c; break;
    }
}

/* ---------------------------------------------------------------- normals */
/* the 2 normals of draw d (Box-Muller on one Philox block) */
DG_FN void dg_normal_pair(uint64_t seed, uint64_t row, uint32_t d, uint32_t tag,
                          double* z0, double* z1) {
    dg_u32x4 r = dg_draw(seed, row, d, tag);
    double u1 = DG_SUB(1.0, dg_u53(r.v[0], r.v[1])); /* (0, 1] */
    double u2 = dg_u53(r.v[2], r.v[3]);              /* [0, 1) */
    double rad = DG_SQRT(DG_MUL(-2.0, dg_ln(u1)));
    double s, c;
    dg_sincos_turns(u2, &s, &c);
    *z0 = DG_MUL(rad, c);
    *z1 = DG_MUL(rad, s);
}

/* z-normalise buf[0..n) in place (FP64, sequential sums) and round to fp32 */
DG_FN void dg_znorm_store(double* buf, int n, float* out) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s = DG_ADD(s, buf[j]);
    double mu = DG_DIV(s, (double)n);
    double v = 0.0;
    for (int j = 0; j < n; ++j) {
        double d = DG_SUB(buf[j], mu);
        v = DG_ADD(v, DG_MUL(d, d));
    }
    double sd = DG_SQRT(DG_DIV(v, (double)n));
    if (!(sd >= 1e-12)) {
        for (int j = 0; j < n; ++j) out[j] = 0.0f;
        return;
    }
    for (int j = 0; j < n; ++j) out[j] = DG_TOF32(DG_DIV(DG_SUB(buf[j], mu), sd));
}

/* one z-normalised random-walk row; buf holds n doubles of scratch */
DG_FN void dg_random_walk_row(uint64_t seed, uint64_t row, int n, double* buf, float* out) {
    double x = 0.0;
    for (int j = 0; j < n; j += 2) {
        double z0, z1;
        dg_normal_pair(seed, row, (uint32_t)(j >> 1), DG_TAG_STEPS, &z0, &z1);
        x = DG_ADD(x, z0);
        buf[j] = x;
        if (j + 1 < n) {
            x = DG_ADD(x, z1);
            buf[j + 1] = x;
        }
    }
    dg_znorm_store(buf, n, out);
}

/* one z-normalised sum-of-3-sinusoids row with N(0, 0.3^2) noise */
DG_FN void dg_sinusoid_row(uint64_t seed, uint64_t row, int n, double* buf, float* out) {
    double f[3], ph[3], a[3];
    for (int c = 0; c < 3; ++c) {
        dg_u32x4 r0 = dg_draw(seed, row, (uint32_t)(2 * c), DG_TAG_PARAMS);
        dg_u32x4 r1 = dg_draw(seed, row, (uint32_t)(2 * c + 1), DG_TAG_PARAMS);
        f[c] = DG_ADD(1.0, DG_MUL(19.0, dg_u53(r0.v[0], r0.v[1])));
        ph[c] = dg_u53(r0.v[2], r0.v[3]);
        a[c] = DG_ADD(0.5, DG_MUL(1.5, dg_u53(r1.v[0], r1.v[1])));
    }
    double z0 = 0.0, z1 = 0.0;
    for (int t = 0; t < n; ++t) {
        if ((t & 1) == 0) dg_normal_pair(seed, row, (uint32_t)(t >> 1), DG_TAG_STEPS, &z0, &z1);
        double v = DG_MUL(0.3, (t & 1) ? z1 : z0);
        for (int c = 0; c < 3; ++c) {
            double turns = DG_ADD(DG_DIV(DG_MUL(f[c], (double)t), (double)n), ph[c]);
            double fl = (double)(int64_t)turns; /* turns >= 0 */
            double fr = DG_SUB(turns, fl);
            double s, co;
            dg_sincos_turns(fr, &s, &co);
            v = DG_ADD(v, DG_MUL(a[c], s));
        }
        buf[t] = v;
    }
    dg_znorm_store(buf, n, out);
}

/* member row + sigma * N(0,1) noise (query id qid, seed qseed), re-normalised */
DG_FN void dg_noisy_row(const float* member, uint64_t qseed, uint64_t qid, int n, double sigma,
                        double* buf, float* out) {
    double z0 = 0.0, z1 = 0.0;
    for (int j = 0; j < n; ++j) {
        if ((j & 1) == 0) dg_normal_pair(qseed, qid, (uint32_t)(j >> 1), DG_TAG_QNOISE, &z0, &z1);
        buf[j] = DG_ADD((double)member[j], DG_MUL(sigma, (j & 1) ? z1 : z0));
    }
    dg_znorm_store(buf, n, out);
}

/* uniform member index in [0, N) for query qid (64-bit multiply-shift) */
DG_FN uint64_t dg_pick_member(uint64_t qseed, uint64_t qid, uint64_t N) {
    dg_u32x4 r = dg_draw(qseed, qid, 0u, DG_TAG_QPICK);
    uint64_t x = ((uint64_t)r.v[0] << 32) | r.v[1];
    /* floor(x * N / 2^64) without 128-bit types */
    uint64_t xh = x >> 32, xl = x & 0xffffffffull, nh = N >> 32, nl = N & 0xffffffffull;
    uint64_t ll = xl * nl, lh = xl * nh, hl = xh * nl, hh = xh * nh;
    uint64_t mid = (ll >> 32) + (lh & 0xffffffffull) + (hl & 0xffffffffull);
    return hh + (lh >> 32) + (hl >> 32) + (mid >> 32);
}

#endif /* ISAX_DG_CORE_H */
