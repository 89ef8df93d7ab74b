/*
 * Oracle sampler for stratified Monte Carlo integration with heuristic tree
 * search (ZMCintegral, arXiv 1902.07916).  TEST INFRASTRUCTURE ONLY: this file
 * is compiled into liboracle_zmc.so, which only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark load.  The product library
 * never links or calls it, and it shares no code with the CUDA path.
 *
 * Plain, slow, obviously correct FP64 C.  It computes, for each requested
 * (cell, trial) pair of one tree level, the direct Monte Carlo sums
 *     S1 = sum_s f(x_s),   S2 = sum_s f(x_s)^2
 * over the n sample points of that trial (Sec. 2.1: each cell's integral is a
 * plain Monte Carlo estimate, repeated over n1 independent trials).  Everything
 * above this step (per-cell mean and standard deviation, threshold, selection,
 * re-splitting, combination) lives in zmc_oracle.py.
 *
 * Random numbers are made at the point of use (Sec. 2.2); the paper names no
 * generator, so the stream is defined here as Philox4x32-10 (Salmon, Moraes,
 * Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11) with key
 * (seed mod 2^32, seed div 2^32), for sample s in [0, n), dimension i in
 * [0, d), trial t, work-list slot q and level L (1-based):
 *   FP64 stream: sample s reads 32-bit word (s mod 4) of the block with
 *                counter ((s div 4) d + i, t, q, L), u = (w + 1/2) 2^-32,
 *                exact in FP64;
 *   FP32 stream: with g = s div 11 and f = s mod 11, sample s reads, of the
 *                pair of blocks with counters (2(g d + i), t, q, L) and
 *                (2(g d + i) + 1, t, q, L) read as 128-bit integers A and B,
 *                the 23-bit field f of A (bits 23 f .. 23 f + 22) for f < 5,
 *                field f - 5 of B for 5 <= f < 10, and for f = 10 the value
 *                (bits 115..127 of A) + 2^13 (bits 115..124 of B);
 *                u = (field + 1/2) 2^-23, exact in FP32.
 * Both uniforms lie strictly inside (0, 1).
 * Sample:  x_i = lo_i + (c_i + u) * w_i, with c_i the cell's lattice
 *          coordinate at level L and w_i = (hi_i - lo_i) / k^L.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- Philox */

/* Round multipliers and key increments of Philox4x32 (SC'11, Sec. 5). */
#define PHILOX_MUL_A 0xD2511F53u
#define PHILOX_MUL_B 0xCD9E8D57u
#define PHILOX_WEYL_A 0x9E3779B9u /* floor(2^32 * (golden ratio - 1)) */
#define PHILOX_WEYL_B 0xBB67AE85u /* floor(2^32 * (sqrt(3) - 1))      */

/* One Philox4x32 round: two 32x32->64 products, the high halves XORed with
 * the other two counter words and the round key, words permuted. */
static void philox_round(uint32_t c[4], const uint32_t key[2]) {
    uint64_t p0 = (uint64_t)PHILOX_MUL_A * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)PHILOX_MUL_B * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ key[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ key[1];
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

/* Philox4x32-10: ten rounds, the key bumped by the Weyl increments between
 * rounds.  out may alias ctr. */
void zmc_oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key_in[2],
                              uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t key[2] = {key_in[0], key_in[1]};
    for (int r = 0; r < 10; ++r) {
        philox_round(c, key);
        key[0] += PHILOX_WEYL_A;
        key[1] += PHILOX_WEYL_B;
    }
    memcpy(out, c, sizeof c);
}

/* The uniform of one 32-bit word, FP64 reading: (w + 1/2) / 2^32. */
double zmc_oracle_uniform64(uint32_t w) {
    return ((double)w + 0.5) * (1.0 / 4294967296.0);
}

/* The FP32-evaluation stream packs five 23-bit fields into each block: read
 * the block as the 128-bit integer B = w0 + 2^32 w1 + 2^64 w2 + 2^96 w3;
 * field f (0..4) is bits [23 f, 23 f + 23) of B, and its uniform is
 * (field + 1/2) / 2^23. */
uint32_t zmc_oracle_field23(const uint32_t w[4], int f) {
    uint32_t out = 0;
    for (int b = 0; b < 23; ++b) {
        const int bit = 23 * f + b;
        const uint32_t v = (w[bit / 32] >> (bit % 32)) & 1u;
        out |= v << b;
    }
    return out;
}

double zmc_oracle_field_uniform(uint32_t field) {
    return ((double)field + 0.5) * (1.0 / 8388608.0);
}

/* Bits [lo, lo + len) of a block read as the 128-bit integer above. */
static uint32_t block_bits(const uint32_t w[4], int lo, int len) {
    uint32_t out = 0;
    for (int b = 0; b < len; ++b) {
        const int bit = lo + b;
        out |= ((w[bit / 32] >> (bit % 32)) & 1u) << b;
    }
    return out;
}

/* Field f (0..10) of a pair of blocks (a, b) in the FP32 stream. */
uint32_t zmc_oracle_pair_field(const uint32_t a[4], const uint32_t b[4], int f) {
    if (f < 5) return zmc_oracle_field23(a, f);
    if (f < 10) return zmc_oracle_field23(b, f - 5);
    return block_bits(a, 115, 13) | (block_bits(b, 115, 10) << 13);
}

/* The uniform of sample s, dimension i, of the (level, slot, trial) stream
 * (the definitions in the header comment). */
static double stream_uniform(const uint32_t key[2], int level, uint32_t slot, uint32_t trial,
                             int d, int fp32, int64_t s, int i) {
    uint32_t w[4];
    if (!fp32) {
        uint32_t ctr[4] = {(uint32_t)((s / 4) * d + i), trial, slot, (uint32_t)level};
        zmc_oracle_philox4x32_10(ctr, key, w);
        return zmc_oracle_uniform64(w[s % 4]);
    }
    uint32_t w2[4];
    uint32_t ca[4] = {(uint32_t)(2 * ((s / 11) * d + i)), trial, slot, (uint32_t)level};
    uint32_t cb[4] = {ca[0] + 1u, trial, slot, (uint32_t)level};
    zmc_oracle_philox4x32_10(ca, key, w);
    zmc_oracle_philox4x32_10(cb, key, w2);
    return zmc_oracle_field_uniform(zmc_oracle_pair_field(w, w2, (int)(s % 11)));
}

/* Uniforms of the (level, slot, trial) stream for points [s0, s0 + count),
 * all d dimensions, point-major: out[(s - s0)*d + i]; fp32 selects the FP32
 * stream. */
void zmc_oracle_stream_uniforms(uint64_t seed, int level, uint32_t slot, uint32_t trial,
                                int d, int fp32, int64_t s0, int64_t count, double* out) {
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    for (int64_t s = s0; s < s0 + count; ++s)
        for (int i = 0; i < d; ++i)
            out[(s - s0) * d + i] = stream_uniform(key, level, slot, trial, d, fp32, s, i);
}

/* Fill `out` with the words of the (level, slot, trial) stream for samples
 * [s0, s0 + count) and all d dimensions, sample-major: out[(s - s0)*d + i]. */
void zmc_oracle_stream_words(uint64_t seed, int level, uint32_t slot,
                             uint32_t trial, int d, int64_t s0, int64_t count,
                             uint32_t* out) {
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    for (int64_t s = s0; s < s0 + count; ++s) {
        for (int i = 0; i < d; ++i) {
            uint32_t ctr[4] = {(uint32_t)((s / 4) * d + i), trial, slot,
                               (uint32_t)level};
            uint32_t w[4];
            zmc_oracle_philox4x32_10(ctr, key, w);
            out[(s - s0) * d + i] = w[s % 4];
        }
    }
}

/* ------------------------------------------------------------ integrands */

enum {
    ORC_CONSTANT = 0,      /* f = p0                                      */
    ORC_LINEAR = 1,        /* f = p0 + sum_i p_{1+i} x_i                   */
    ORC_SIN_SUM = 2,       /* f1 of Eq. (1): sin(sum_i x_i)                */
    ORC_GAUSS_NORM = 3,    /* f2 of Eq. (2), width p0                      */
    ORC_GENZ_OSC = 4,      /* cos(2 pi p0 + sum_i a_i x_i), a = p[1..d]    */
    ORC_GENZ_PRODPEAK = 5, /* prod_i 1/(a_i^-2 + (x_i-u_i)^2)              */
    ORC_GENZ_GAUSS = 6,    /* exp(-sum_i a_i^2 (x_i-u_i)^2)                */
    ORC_GENZ_CORNER = 7    /* (1 + sum_i a_i x_i)^-(d+1)                   */
};

static const double ORC_PI = 3.14159265358979323846;

/* The integrand at one point, FP64, written out as its formula. */
double zmc_oracle_integrand(int id, int d, const double* x, const double* p) {
    switch (id) {
    case ORC_CONSTANT:
        return p[0];
    case ORC_LINEAR: {
        double v = p[0];
        for (int i = 0; i < d; ++i) v += p[1 + i] * x[i];
        return v;
    }
    case ORC_SIN_SUM: {
        double s = 0.0;
        for (int i = 0; i < d; ++i) s += x[i];
        return sin(s);
    }
    case ORC_GAUSS_NORM: {
        /* Eq. (2) for d dimensions: (sqrt(2 pi) sigma)^-d exp(-|x|^2/(2 sigma^2)) */
        double sigma = p[0];
        double r2 = 0.0;
        for (int i = 0; i < d; ++i) r2 += x[i] * x[i];
        double norm = pow(sqrt(2.0 * ORC_PI) * sigma, -(double)d);
        return norm * exp(-r2 / (2.0 * sigma * sigma));
    }
    case ORC_GENZ_OSC: {
        double s = 2.0 * ORC_PI * p[0];
        for (int i = 0; i < d; ++i) s += p[1 + i] * x[i];
        return cos(s);
    }
    case ORC_GENZ_PRODPEAK: {
        double v = 1.0;
        for (int i = 0; i < d; ++i) {
            double a = p[i], u = p[d + i];
            v *= 1.0 / (1.0 / (a * a) + (x[i] - u) * (x[i] - u));
        }
        return v;
    }
    case ORC_GENZ_GAUSS: {
        double s = 0.0;
        for (int i = 0; i < d; ++i) {
            double a = p[i], u = p[d + i];
            s += a * a * (x[i] - u) * (x[i] - u);
        }
        return exp(-s);
    }
    case ORC_GENZ_CORNER: {
        double s = 1.0;
        for (int i = 0; i < d; ++i) s += p[i] * x[i];
        return pow(s, -(double)(d + 1));
    }
    default:
        return NAN;
    }
}

/* ------------------------------------------------------- (cell, trial) sums */

typedef struct {
    uint64_t seed;
    int level, d, integrand, fp32_uniforms;
    const double *lo, *width, *params;
    int64_t n;
    int trials;
    int64_t n_cells;
    const uint32_t* slots;   /* work-list slot q of each requested cell      */
    const int64_t* coords;   /* n_cells x d lattice coordinates at `level`   */
    double* out;             /* n_cells x trials x 2: (S1, S2)               */
    int64_t next;            /* next (cell, trial) job, claimed under lock   */
    pthread_mutex_t lock;
} sums_job;

static void one_cell_trial(const sums_job* J, int64_t cell, int trial) {
    const int d = J->d;
    uint32_t key[2] = {(uint32_t)(J->seed & 0xFFFFFFFFu),
                       (uint32_t)(J->seed >> 32)};
    double x[64];
    uint32_t words[64][2][4];
    double S1 = 0.0, S2 = 0.0;
    const int64_t* c = J->coords + cell * d;
    /* points per group: 4 words of one block (FP64 stream) or 11 fields of a
       pair of blocks (FP32 stream) */
    const int G = J->fp32_uniforms ? 11 : 4, B = J->fp32_uniforms ? 2 : 1;
    for (int64_t s = 0; s < J->n; ++s) {
        if (s % G == 0) {
            /* the d (pairs of) Philox blocks that carry samples s .. s+G-1 */
            for (int i = 0; i < d; ++i)
                for (int b = 0; b < B; ++b) {
                    uint32_t ctr[4] = {(uint32_t)(B * ((s / G) * d + i) + b), (uint32_t)trial,
                                       J->slots[cell], (uint32_t)J->level};
                    zmc_oracle_philox4x32_10(ctr, key, words[i][b]);
                }
        }
        for (int i = 0; i < d; ++i) {
            double u = J->fp32_uniforms
                           ? zmc_oracle_field_uniform(
                                 zmc_oracle_pair_field(words[i][0], words[i][1], (int)(s % G)))
                           : zmc_oracle_uniform64(words[i][0][s % G]);
            x[i] = J->lo[i] + ((double)c[i] + u) * J->width[i];
        }
        double f = zmc_oracle_integrand(J->integrand, d, x, J->params);
        S1 += f;
        S2 += f * f;
    }
    J->out[(cell * J->trials + trial) * 2 + 0] = S1;
    J->out[(cell * J->trials + trial) * 2 + 1] = S2;
}

static void* sums_worker(void* arg) {
    sums_job* J = (sums_job*)arg;
    const int64_t total = J->n_cells * J->trials;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int64_t job = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (job >= total) break;
        one_cell_trial(J, job / J->trials, (int)(job % J->trials));
    }
    return NULL;
}

/* For each requested cell of one level and each trial, the sums (S1, S2).
 * width[i] = (hi_i - lo_i) / k^level.  Returns 0, or -1 on bad arguments.
 * fp32_uniforms selects the FP32-evaluation stream (eleven 23-bit fields per
 * pair of blocks): the points the FP32 modes sample; everything else stays
 * FP64. */
int zmc_oracle_cell_sums(uint64_t seed, int level, int d, const double* lo,
                         const double* width, int64_t n, int trials,
                         int integrand, const double* params, int64_t n_cells,
                         const uint32_t* slots, const int64_t* coords,
                         int fp32_uniforms, int threads, double* out) {
    if (d < 1 || d > 64 || n < 1 || trials < 1 || n_cells < 0 || threads < 1)
        return -1;
    sums_job J;
    J.seed = seed; J.level = level; J.d = d; J.integrand = integrand;
    J.fp32_uniforms = fp32_uniforms;
    J.lo = lo; J.width = width; J.params = params;
    J.n = n; J.trials = trials; J.n_cells = n_cells;
    J.slots = slots; J.coords = coords; J.out = out; J.next = 0;
    pthread_mutex_init(&J.lock, NULL);
    if (threads > 256) threads = 256;
    pthread_t tid[256];
    int started = 0;
    for (int i = 0; i < threads; ++i)
        if (pthread_create(&tid[i], NULL, sums_worker, &J) == 0) ++started;
    if (started == 0) sums_worker(&J);
    for (int i = 0; i < started; ++i) pthread_join(tid[i], NULL);
    pthread_mutex_destroy(&J.lock);
    return 0;
}
