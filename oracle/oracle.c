/*
 * oracle.c — the CPU oracle for the prefix sum (scan).  TEST INFRASTRUCTURE.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this code.  The product path (the CUDA library and its Python binding)
 * never calls it, and this file includes nothing from the product.
 *
 * Every function is the plain, sequential definition of the operation, written
 * for obviousness, not speed: one loop carrying a running total, exactly as the
 * paper states the problem (Section 1, Introduction: an inclusive scan outputs
 * [a0, a0+a1, ..., a0+...+a_{n-1}]; an exclusive scan drops the last of those
 * and puts the identity, 0, first; the baseline algorithm walks the input
 * once, adding each element to a running total and writing the total out).
 *
 * Readings where the paper is silent:
 *  - Integer overflow (the paper only uses fp32, Section 4.1): two's-complement
 *    wraparound.  The running total is kept in uint32_t / uint64_t, where C
 *    defines wraparound, and reinterpreted.
 *  - Floating-point inputs: the paper notes that a parallel float scan differs
 *    from the sequential one because float addition is not associative
 *    (Section 1.1, Related Work).  The reference result for float (and double)
 *    input is therefore the prefix sum accumulated in double with Neumaier's
 *    compensated summation (Neumaier 1974), written as double.  A plain-double
 *    variant is kept to cross-check it.
 *  - Segmented scans (not in the paper; the same definition restarted at every
 *    segment start): segment s covers [offsets[s], offsets[s+1]).
 *  - The reverse (suffix) scan used by the gradient: y_i = sum_{k >= i} a_k
 *    (inclusive) or sum_{k > i} a_k (exclusive), per row.
 *  - Other associative operators (Section 1 defines the scan for +; the same
 *    definition holds for any associative operator): the running maximum and
 *    minimum.  An exclusive scan starts from the operator's identity
 *    (INT32_MIN / INT64_MIN / 0 / -inf for max, INT32_MAX / INT64_MAX /
 *    UINT32_MAX / +inf for min, for int32 / int64 / uint32 / fp32).  fp32 max
 *    and min are C's fmaxf / fminf (IEEE maxNum / minNum: a NaN operand yields
 *    the other one).  Segmented maxima and minima restart at every segment
 *    start, like the segmented sums.
 *  - Unsigned 32-bit sums: the same modular running total as int32 (the
 *    bits of an int32 and a uint32 sum are the same); it has its own loop so
 *    that the unsigned entry points are checked against an unsigned
 *    definition.
 *  - Stream compaction (an application of the scan that Section 1 lists):
 *    copy, in order, the elements whose keep flag is nonzero; the number kept
 *    is the total of the flags.  Elements are moved as 4-byte words.
 */
#include <math.h>
#include <stdint.h>

/* ---- integer scans (Section 1 definition, modular arithmetic) ----------- */

void oracle_scan_i32(const int32_t* a, int32_t* y, int64_t n, int exclusive) {
    uint32_t run = 0;
    for (int64_t k = 0; k < n; ++k) {
        uint32_t ak = (uint32_t)a[k];
        if (exclusive) {
            y[k] = (int32_t)run;
            run += ak;
        } else {
            run += ak;
            y[k] = (int32_t)run;
        }
    }
}

void oracle_scan_i64(const int64_t* a, int64_t* y, int64_t n, int exclusive) {
    uint64_t run = 0;
    for (int64_t k = 0; k < n; ++k) {
        uint64_t ak = (uint64_t)a[k];
        if (exclusive) {
            y[k] = (int64_t)run;
            run += ak;
        } else {
            run += ak;
            y[k] = (int64_t)run;
        }
    }
}

/* Total of a (modular), computed by its own loop: the last inclusive output
 * must equal it (Section 2.1: the last element of a partition's prefix sum is
 * the partition total). */
int32_t oracle_reduce_i32(const int32_t* a, int64_t n) {
    uint32_t s = 0;
    for (int64_t k = 0; k < n; ++k) s += (uint32_t)a[k];
    return (int32_t)s;
}

int64_t oracle_reduce_i64(const int64_t* a, int64_t n) {
    uint64_t s = 0;
    for (int64_t k = 0; k < n; ++k) s += (uint64_t)a[k];
    return (int64_t)s;
}

/* ---- floating point: the FP64 reference -------------------------------- */

/* Neumaier's improved Kahan summation: s holds the rounded running sum, c the
 * accumulated rounding errors; the reported prefix is s + c. */
typedef struct {
    double s, c;
} neum_t;

static inline void neum_add(neum_t* acc, double x) {
    double t = acc->s + x;
    if (fabs(acc->s) >= fabs(x))
        acc->c += (acc->s - t) + x;
    else
        acc->c += (x - t) + acc->s;
    acc->s = t;
}

void oracle_scan_f32_ref(const float* a, double* y, int64_t n, int exclusive) {
    neum_t acc = {0.0, 0.0};
    for (int64_t k = 0; k < n; ++k) {
        if (exclusive) {
            y[k] = acc.s + acc.c;
            neum_add(&acc, (double)a[k]);
        } else {
            neum_add(&acc, (double)a[k]);
            y[k] = acc.s + acc.c;
        }
    }
}

void oracle_scan_f64_ref(const double* a, double* y, int64_t n, int exclusive) {
    neum_t acc = {0.0, 0.0};
    for (int64_t k = 0; k < n; ++k) {
        if (exclusive) {
            y[k] = acc.s + acc.c;
            neum_add(&acc, a[k]);
        } else {
            neum_add(&acc, a[k]);
            y[k] = acc.s + acc.c;
        }
    }
}

/* Plain double accumulation, kept only to cross-check the compensated one. */
void oracle_scan_f32_plain_f64(const float* a, double* y, int64_t n, int exclusive) {
    double run = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        if (exclusive) {
            y[k] = run;
            run += (double)a[k];
        } else {
            run += (double)a[k];
            y[k] = run;
        }
    }
}

/* Prefix sums of |a_k| in double: the denominator sum_{i<=k} |a_i| of the
 * error metric (exclusive: sum_{i<k} |a_i|). */
void oracle_abs_scan_f32(const float* a, double* y, int64_t n, int exclusive) {
    neum_t acc = {0.0, 0.0};
    for (int64_t k = 0; k < n; ++k) {
        if (exclusive) {
            y[k] = acc.s + acc.c;
            neum_add(&acc, fabs((double)a[k]));
        } else {
            neum_add(&acc, fabs((double)a[k]));
            y[k] = acc.s + acc.c;
        }
    }
}

/* ---- segmented scans ---------------------------------------------------- */

/* The Section 1 definition applied to each segment [offsets[s], offsets[s+1])
 * on its own.  Elements outside [offsets[0], offsets[S]) are not touched. */
void oracle_seg_scan_i32(const int32_t* a, int32_t* y, const int64_t* offsets,
                         int64_t num_segments, int exclusive) {
    for (int64_t s = 0; s < num_segments; ++s) {
        int64_t b = offsets[s], e = offsets[s + 1];
        if (e > b) oracle_scan_i32(a + b, y + b, e - b, exclusive);
    }
}

void oracle_seg_scan_i64(const int64_t* a, int64_t* y, const int64_t* offsets,
                         int64_t num_segments, int exclusive) {
    for (int64_t s = 0; s < num_segments; ++s) {
        int64_t b = offsets[s], e = offsets[s + 1];
        if (e > b) oracle_scan_i64(a + b, y + b, e - b, exclusive);
    }
}

void oracle_seg_scan_f32_ref(const float* a, double* y, const int64_t* offsets,
                             int64_t num_segments, int exclusive) {
    for (int64_t s = 0; s < num_segments; ++s) {
        int64_t b = offsets[s], e = offsets[s + 1];
        if (e > b) oracle_scan_f32_ref(a + b, y + b, e - b, exclusive);
    }
}

void oracle_seg_abs_scan_f32(const float* a, double* y, const int64_t* offsets,
                             int64_t num_segments, int exclusive) {
    for (int64_t s = 0; s < num_segments; ++s) {
        int64_t b = offsets[s], e = offsets[s + 1];
        if (e > b) oracle_abs_scan_f32(a + b, y + b, e - b, exclusive);
    }
}

/* ---- reverse (suffix) scans per row: the gradient of a row-wise scan ---- */

/* y[r, i] = sum_{k >= i} a[r, k]  (exclusive: k > i), row-major rows x cols,
 * accumulated from the end of each row towards its start in double with the
 * same compensated summation. */
void oracle_rows_suffix_f32_ref(const float* a, double* y, int64_t rows, int64_t cols,
                                int exclusive) {
    for (int64_t r = 0; r < rows; ++r) {
        const float* ar = a + r * cols;
        double* yr = y + r * cols;
        neum_t acc = {0.0, 0.0};
        for (int64_t i = cols - 1; i >= 0; --i) {
            if (exclusive) {
                yr[i] = acc.s + acc.c;
                neum_add(&acc, (double)ar[i]);
            } else {
                neum_add(&acc, (double)ar[i]);
                yr[i] = acc.s + acc.c;
            }
        }
    }
}

void oracle_rows_suffix_f64_ref(const double* a, double* y, int64_t rows, int64_t cols,
                                int exclusive) {
    for (int64_t r = 0; r < rows; ++r) {
        const double* ar = a + r * cols;
        double* yr = y + r * cols;
        neum_t acc = {0.0, 0.0};
        for (int64_t i = cols - 1; i >= 0; --i) {
            if (exclusive) {
                yr[i] = acc.s + acc.c;
                neum_add(&acc, ar[i]);
            } else {
                neum_add(&acc, ar[i]);
                yr[i] = acc.s + acc.c;
            }
        }
    }
}

void oracle_rows_suffix_abs_f32(const float* a, double* y, int64_t rows, int64_t cols,
                                int exclusive) {
    for (int64_t r = 0; r < rows; ++r) {
        const float* ar = a + r * cols;
        double* yr = y + r * cols;
        neum_t acc = {0.0, 0.0};
        for (int64_t i = cols - 1; i >= 0; --i) {
            if (exclusive) {
                yr[i] = acc.s + acc.c;
                neum_add(&acc, fabs((double)ar[i]));
            } else {
                neum_add(&acc, fabs((double)ar[i]));
                yr[i] = acc.s + acc.c;
            }
        }
    }
}

/* ---- running maximum / minimum (same definition, another operator) ------- */

void oracle_scan_max_i32(const int32_t* a, int32_t* y, int64_t n, int exclusive) {
    int32_t run = INT32_MIN;
    for (int64_t k = 0; k < n; ++k) {
        if (exclusive) y[k] = run;
        if (a[k] > run) run = a[k];
        if (!exclusive) y[k] = run;
    }
}

void oracle_scan_min_i32(const int32_t* a, int32_t* y, int64_t n, int exclusive) {
    int32_t run = INT32_MAX;
    for (int64_t k = 0; k < n; ++k) {
        if (exclusive) y[k] = run;
        if (a[k] < run) run = a[k];
        if (!exclusive) y[k] = run;
    }
}

void oracle_scan_max_f32(const float* a, float* y, int64_t n, int exclusive) {
    float run = -INFINITY;
    for (int64_t k = 0; k < n; ++k) {
        if (exclusive) y[k] = run;
        run = fmaxf(run, a[k]);
        if (!exclusive) y[k] = run;
    }
}

void oracle_scan_min_f32(const float* a, float* y, int64_t n, int exclusive) {
    float run = INFINITY;
    for (int64_t k = 0; k < n; ++k) {
        if (exclusive) y[k] = run;
        run = fminf(run, a[k]);
        if (!exclusive) y[k] = run;
    }
}

void oracle_scan_max_i64(const int64_t* a, int64_t* y, int64_t n, int exclusive) {
    int64_t run = INT64_MIN;
    for (int64_t k = 0; k < n; ++k) {
        if (exclusive) y[k] = run;
        if (a[k] > run) run = a[k];
        if (!exclusive) y[k] = run;
    }
}

void oracle_scan_min_i64(const int64_t* a, int64_t* y, int64_t n, int exclusive) {
    int64_t run = INT64_MAX;
    for (int64_t k = 0; k < n; ++k) {
        if (exclusive) y[k] = run;
        if (a[k] < run) run = a[k];
        if (!exclusive) y[k] = run;
    }
}

void oracle_scan_max_u32(const uint32_t* a, uint32_t* y, int64_t n, int exclusive) {
    uint32_t run = 0;
    for (int64_t k = 0; k < n; ++k) {
        if (exclusive) y[k] = run;
        if (a[k] > run) run = a[k];
        if (!exclusive) y[k] = run;
    }
}

void oracle_scan_min_u32(const uint32_t* a, uint32_t* y, int64_t n, int exclusive) {
    uint32_t run = UINT32_MAX;
    for (int64_t k = 0; k < n; ++k) {
        if (exclusive) y[k] = run;
        if (a[k] < run) run = a[k];
        if (!exclusive) y[k] = run;
    }
}

/* ---- unsigned 32-bit sums ------------------------------------------------ */

void oracle_scan_u32(const uint32_t* a, uint32_t* y, int64_t n, int exclusive) {
    uint32_t run = 0;
    for (int64_t k = 0; k < n; ++k) {
        if (exclusive) {
            y[k] = run;
            run += a[k];
        } else {
            run += a[k];
            y[k] = run;
        }
    }
}

/* ---- segmented running maximum / minimum --------------------------------- */

void oracle_seg_scan_max_i32(const int32_t* a, int32_t* y, const int64_t* offsets,
                             int64_t num_segments, int exclusive) {
    for (int64_t s = 0; s < num_segments; ++s) {
        int64_t b = offsets[s], e = offsets[s + 1];
        if (e > b) oracle_scan_max_i32(a + b, y + b, e - b, exclusive);
    }
}

void oracle_seg_scan_min_i32(const int32_t* a, int32_t* y, const int64_t* offsets,
                             int64_t num_segments, int exclusive) {
    for (int64_t s = 0; s < num_segments; ++s) {
        int64_t b = offsets[s], e = offsets[s + 1];
        if (e > b) oracle_scan_min_i32(a + b, y + b, e - b, exclusive);
    }
}

void oracle_seg_scan_max_f32(const float* a, float* y, const int64_t* offsets,
                             int64_t num_segments, int exclusive) {
    for (int64_t s = 0; s < num_segments; ++s) {
        int64_t b = offsets[s], e = offsets[s + 1];
        if (e > b) oracle_scan_max_f32(a + b, y + b, e - b, exclusive);
    }
}

void oracle_seg_scan_min_f32(const float* a, float* y, const int64_t* offsets,
                             int64_t num_segments, int exclusive) {
    for (int64_t s = 0; s < num_segments; ++s) {
        int64_t b = offsets[s], e = offsets[s + 1];
        if (e > b) oracle_scan_min_f32(a + b, y + b, e - b, exclusive);
    }
}

/* ---- stream compaction --------------------------------------------------- */

int64_t oracle_compact_u32(const uint32_t* in, const uint8_t* flags, uint32_t* out, int64_t n) {
    int64_t j = 0;
    for (int64_t i = 0; i < n; ++i)
        if (flags[i] != 0) out[j++] = in[i];
    return j;
}
