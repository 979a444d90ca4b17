/*
 * synth.c — seeded synthetic inputs shared by the CPU oracle, the GPU tests
 * and the benchmark.
 *
 * This file holds no prefix-sum arithmetic: it only draws numbers.  The paper
 * measures on "random data" (Section 4.1, experimental setup) without naming a
 * generator, so the generator is fixed here:
 *
 *   element i of stream (seed, stream) is  x_i = mix64(key + (i + 1) * GAMMA),
 *   key = seed * 2^32 + stream,
 *
 * where mix64/GAMMA are the finaliser and increment of SplitMix64 (Steele, Lea
 * and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014).
 * With key = 0 the sequence is the canonical SplitMix64 stream seeded with 0.
 * Being counter based, any element can be drawn independently, so large arrays
 * are filled by several host threads with a reproducible result.
 *
 * Derived distributions (all exact, no libm except for the normal draw and the
 * log-uniform segment lengths):
 *   uniform integer in [0, m), m <= 2^32 :  ((x >> 32) * m) >> 32
 *   uniform float in [0, 1) on the 2^-24 grid :  (x >> 40) * 2^-24
 *   standard normal (Box-Muller, in double, rounded once to float):
 *       u1 = ((x_{2i} >> 11) + 1) * 2^-53 in (0, 1],  u2 = (x_{2i+1} >> 11) * 2^-53
 *       z  = sqrt(-2 ln u1) * cos(2 pi u2)
 *   log-uniform segment length in [1, 2^e]:  floor(2^(e * u)), u = (x >> 11) * 2^-53,
 *       clamped to [1, 2^e].
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <unistd.h>

#define SYNTH_GAMMA 0x9e3779b97f4a7c15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static inline uint64_t draw(uint64_t key, uint64_t i) {
    return mix64(key + (i + 1) * SYNTH_GAMMA);
}

static inline uint64_t make_key(uint64_t seed, uint64_t stream) {
    return (seed << 32) + (stream & 0xffffffffULL);
}

/* ---- element kernels ---------------------------------------------------- */

enum { K_RAW = 0, K_I32 = 1, K_I64 = 2, K_F32_UNIT = 3, K_F32_NORMAL = 4, K_F64_NORMAL = 5 };

typedef struct {
    int kind;
    uint64_t key;
    uint64_t m;
    void* out;
    int64_t begin, end; /* element range [begin, end) */
    int64_t first;      /* index of out[0] in the stream */
} job_t;

static void fill_range(const job_t* j) {
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t i = j->begin; i < j->end; ++i) {
        uint64_t c = (uint64_t)(j->first + i);
        switch (j->kind) {
        case K_RAW:
            ((uint64_t*)j->out)[i] = draw(j->key, c);
            break;
        case K_I32: {
            uint64_t x = draw(j->key, c);
            ((uint32_t*)j->out)[i] = (uint32_t)(((x >> 32) * j->m) >> 32);
            break;
        }
        case K_I64: {
            uint64_t x = draw(j->key, c);
            ((uint64_t*)j->out)[i] = ((x >> 32) * j->m) >> 32;
            break;
        }
        case K_F32_UNIT: {
            uint64_t x = draw(j->key, c);
            ((float*)j->out)[i] = (float)((double)(x >> 40) * 0x1p-24);
            break;
        }
        case K_F32_NORMAL:
        case K_F64_NORMAL: {
            uint64_t x1 = draw(j->key, 2 * c), x2 = draw(j->key, 2 * c + 1);
            double u1 = (double)((x1 >> 11) + 1) * 0x1p-53;
            double u2 = (double)(x2 >> 11) * 0x1p-53;
            double z = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
            if (j->kind == K_F32_NORMAL)
                ((float*)j->out)[i] = (float)z;
            else
                ((double*)j->out)[i] = z;
            break;
        }
        }
    }
}

static void* fill_thread(void* arg) {
    fill_range((const job_t*)arg);
    return NULL;
}

static void fill(int kind, uint64_t seed, uint64_t stream, uint64_t m, void* out, int64_t n,
                 int64_t first) {
    if (n <= 0) return;
    job_t base = {kind, make_key(seed, stream), m, out, 0, n, first};
    long ncpu = sysconf(_SC_NPROCESSORS_ONLN);
    int nt = (int)(ncpu < 1 ? 1 : (ncpu > 32 ? 32 : ncpu));
    if (n < (1 << 20) || nt == 1) {
        fill_range(&base);
        return;
    }
    pthread_t th[32];
    job_t jobs[32];
    int started[32] = {0};
    int64_t chunk = (n + nt - 1) / nt;
    for (int t = 0; t < nt; ++t) {
        jobs[t] = base;
        jobs[t].begin = (int64_t)t * chunk;
        jobs[t].end = jobs[t].begin + chunk < n ? jobs[t].begin + chunk : n;
        if (jobs[t].begin >= jobs[t].end) continue;
        if (pthread_create(&th[t], NULL, fill_thread, &jobs[t]) == 0)
            started[t] = 1;
        else
            fill_range(&jobs[t]);
    }
    for (int t = 0; t < nt; ++t)
        if (started[t]) pthread_join(th[t], NULL);
}

/* ---- exported API -------------------------------------------------------- */

/* Raw 64-bit draws x_first .. x_{first+n-1}. */
void synth_raw_u64(uint64_t seed, uint64_t stream, uint64_t* out, int64_t n, int64_t first) {
    fill(K_RAW, seed, stream, 0, out, n, first);
}

/* Uniform integers in [0, m), 1 <= m <= 2^32, stored as int32 bit patterns. */
void synth_uniform_i32(uint64_t seed, uint64_t stream, uint64_t m, int32_t* out, int64_t n) {
    fill(K_I32, seed, stream, m, out, n, 0);
}

/* Uniform integers in [0, m), 1 <= m <= 2^32, stored as int64. */
void synth_uniform_i64(uint64_t seed, uint64_t stream, uint64_t m, int64_t* out, int64_t n) {
    fill(K_I64, seed, stream, m, out, n, 0);
}

/* Uniform floats k * 2^-24, k uniform in [0, 2^24). */
void synth_unit_f32(uint64_t seed, uint64_t stream, float* out, int64_t n) {
    fill(K_F32_UNIT, seed, stream, 0, out, n, 0);
}

/* Standard normal floats (Box-Muller in double, rounded once). */
void synth_normal_f32(uint64_t seed, uint64_t stream, float* out, int64_t n) {
    fill(K_F32_NORMAL, seed, stream, 0, out, n, 0);
}

/* Standard normal doubles (Box-Muller). */
void synth_normal_f64(uint64_t seed, uint64_t stream, double* out, int64_t n) {
    fill(K_F64_NORMAL, seed, stream, 0, out, n, 0);
}

/* Segment boundaries: num_segments lengths, log-uniform in [1, 2^max_log2],
 * written as a CSR offsets array of num_segments + 1 entries starting at 0.
 * Returns the total length offsets[num_segments]. */
int64_t synth_segment_offsets(uint64_t seed, uint64_t stream, int64_t num_segments, int max_log2,
                              int64_t* offsets) {
    uint64_t key = make_key(seed, stream);
    double cap = ldexp(1.0, max_log2);
    offsets[0] = 0;
    for (int64_t s = 0; s < num_segments; ++s) {
        double u = (double)(draw(key, (uint64_t)s) >> 11) * 0x1p-53;
        double len = floor(exp2((double)max_log2 * u));
        if (len < 1.0) len = 1.0;
        if (len > cap) len = cap;
        offsets[s + 1] = offsets[s] + (int64_t)len;
    }
    return offsets[num_segments];
}
