"""Pins for the CPU oracle (no GPU).

Each check ties the oracle to something other than itself: the hand-worked
definition example, closed forms, brute force with Python integers, library
routines for special cases (numpy cumsum in exact integer arithmetic, math.fsum
for correctly rounded float sums, a dense matrix product for the Jacobian), and
invariants from the paper (Section 1 definition; Section 2.1: the last element
of a partition's prefix sum is the partition total).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden

M32 = 1 << 32


def to_i32(v):
    v %= M32
    return v - M32 if v >= 1 << 31 else v


def brute_scan(a, exclusive=False, wrap=None):
    """O(n^2) brute force: every output summed from scratch with Python ints."""
    out = []
    for k in range(len(a)):
        terms = a[:k] if exclusive else a[:k + 1]
        s = sum(int(t) for t in terms)
        out.append(wrap(s) if wrap else s)
    return out


# ---- the definition example ---------------------------------------------

def test_golden_definition_example():
    g = read_golden("definition_example.txt")
    a = np.array(g["input"])
    assert oracle.scan_i32(a).tolist() == g["inclusive"]
    assert oracle.scan_i32(a, exclusive=True).tolist() == g["exclusive"]
    assert oracle.scan_i64(a).tolist() == g["inclusive"]
    assert oracle.scan_i64(a, exclusive=True).tolist() == g["exclusive"]
    assert oracle.scan_f32_ref(a).tolist() == [float(v) for v in g["inclusive"]]
    assert oracle.scan_f32_ref(a, exclusive=True).tolist() == [float(v) for v in g["exclusive"]]
    s = oracle.rows_suffix_f32_ref(a.reshape(1, -1)).reshape(-1)
    assert s.tolist() == [float(v) for v in g["suffix_inclusive"]]
    s = oracle.rows_suffix_f32_ref(a.reshape(1, -1), exclusive=True).reshape(-1)
    assert s.tolist() == [float(v) for v in g["suffix_exclusive"]]
    off = np.array(g["offsets"])
    assert oracle.seg_scan_i32(a, off).tolist() == g["seg_inclusive"]
    assert oracle.seg_scan_i32(a, off, exclusive=True).tolist() == g["seg_exclusive"]
    assert oracle.seg_scan_f32_ref(a, off, exclusive=True).tolist() == [
        float(v) for v in g["seg_exclusive"]]


# ---- closed forms ----------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 1000, 1 << 20])
def test_all_ones(n):
    a = np.ones(n, dtype=np.int32)
    k = np.arange(n, dtype=np.int64)
    assert np.array_equal(oracle.scan_i32(a), (k + 1).astype(np.int32))
    assert np.array_equal(oracle.scan_i32(a, True), k.astype(np.int32))
    assert np.array_equal(oracle.scan_i64(a.astype(np.int64)), k + 1)
    assert np.array_equal(oracle.scan_f32_ref(a.astype(np.float32)), (k + 1).astype(np.float64))


def test_triangular_numbers_i64_and_wrapped_i32():
    n = 1 << 20
    i = np.arange(n, dtype=np.int64)
    tri = i * (i + 1) // 2  # < 2^40: exact in int64
    assert np.array_equal(oracle.scan_i64(i), tri)
    # int32: i(i+1)/2 exceeds 2^31 from i ~ 65536 on; the reading is wraparound
    assert np.array_equal(oracle.scan_i32(i.astype(np.int32)),
                          (tri % M32).astype(np.uint32).view(np.int32))
    # exclusive: y_k = (k-1)k/2
    assert np.array_equal(oracle.scan_i64(i, True), (i - 1) * i // 2)


@pytest.mark.parametrize("c", [7, -3, 255, (1 << 31) - 1])
def test_constant_input_wraps(c):
    n = 100_000
    k = np.arange(n, dtype=np.int64)
    want = ((c * (k + 1)) % M32).astype(np.uint32).view(np.int32)
    assert np.array_equal(oracle.scan_i32(np.full(n, c, dtype=np.int32)), want)


def test_i64_wraps_at_2_64():
    a = np.array([(1 << 62), (1 << 62), (1 << 62), (1 << 62), 5], dtype=np.int64)
    want = [brute for brute in brute_scan(a.tolist(), wrap=lambda s: (
        (s + (1 << 63)) % (1 << 64)) - (1 << 63))]
    assert oracle.scan_i64(a).tolist() == want


# ---- brute force on tiny inputs ---------------------------------------------

@pytest.mark.parametrize("n", [0, 1, 2, 3, 17, 31, 32, 33, 64])
@pytest.mark.parametrize("excl", [False, True])
def test_brute_force_i32_i64(n, excl):
    a32 = synth.raw_u64(n, seed=11, stream=n).view(np.int64).astype(np.int32)  # full range
    assert oracle.scan_i32(a32, excl).tolist() == brute_scan(a32.tolist(), excl, to_i32)
    a64 = synth.raw_u64(n, seed=12, stream=n).view(np.int64)
    wrap64 = lambda s: ((s + (1 << 63)) % (1 << 64)) - (1 << 63)
    assert oracle.scan_i64(a64, excl).tolist() == brute_scan(a64.tolist(), excl, wrap64)


@pytest.mark.parametrize("excl", [False, True])
def test_brute_force_float_prefixes_against_fsum(excl):
    """math.fsum gives each prefix correctly rounded; the compensated FP64
    oracle must meet Neumaier's bound |ref - exact| <= 2u|exact| + O(n u^2)
    sum|a| (u = 2^-53).  Wide-range inputs make double accumulation round, so
    plain double accumulation would fail the bound."""
    from test_oracle_mutants import meets_neumaier_bound, wide_range_f32
    n = 1500
    a = wide_range_f32(n, seed=3)
    assert meets_neumaier_bound(oracle.scan_f32_ref(a, excl), a.astype(np.float64), excl)
    assert not meets_neumaier_bound(oracle.scan_f32_plain_f64(a, excl), a.astype(np.float64),
                                    excl)
    a64 = synth.normal_f64(n, seed=3)
    assert meets_neumaier_bound(oracle.scan_f64_ref(a64, excl), a64, excl)
    # the |a| prefix (metric denominator) against fsum of |a|
    den = oracle.abs_scan_f32(a, excl)
    vals = [abs(float(v)) for v in a]
    for k in range(n):
        dexact = math.fsum(vals[:k] if excl else vals[:k + 1])
        assert abs(den[k] - dexact) <= 2.0 ** -52 * dexact


# ---- invariants -------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 5, 4097, 1 << 18])
def test_last_equals_total_and_exclusive_is_shift(n):
    a = synth.uniform_i32(n, 256, seed=0, stream=1)
    inc = oracle.scan_i32(a)
    exc = oracle.scan_i32(a, True)
    assert inc[-1] == oracle.reduce_i32(a)
    assert exc[0] == 0 and np.array_equal(exc[1:], inc[:-1])
    a64 = synth.uniform_i64(n, 1 << 32, seed=0, stream=2)
    inc64 = oracle.scan_i64(a64)
    assert inc64[-1] == oracle.reduce_i64(a64)
    exc64 = oracle.scan_i64(a64, True)
    assert exc64[0] == 0 and np.array_equal(exc64[1:], inc64[:-1])


def test_i32_equals_low_bits_of_wide_scan():
    """The int32 result is the low 32 bits of the same values scanned in int64
    (numpy cumsum, exact here: |partial sums| < 2^63)."""
    n = 300_000
    a = synth.raw_u64(n, seed=5).view(np.int64).astype(np.int32)
    wide = np.cumsum(a.astype(np.int64))
    assert np.array_equal(oracle.scan_i32(a), (wide % M32).astype(np.uint32).view(np.int32))
    assert np.array_equal(oracle.scan_i64(a.astype(np.int64)), wide)


def test_f32_uniform_grid_is_exact():
    """Inputs k * 2^-24 with integer k < 2^24: the true prefix is 2^-24 times an
    integer prefix (< 2^53), exactly representable in double, so the FP64
    oracle must match the integer scan bit for bit."""
    n = 1 << 22
    a = synth.unit_f32(n, seed=0, stream=7)
    k = (a.astype(np.float64) * 2.0 ** 24).astype(np.int64)
    assert np.array_equal(k.astype(np.float64) * 2.0 ** -24, a.astype(np.float64))
    want = np.cumsum(k).astype(np.float64) * 2.0 ** -24
    assert np.array_equal(oracle.scan_f32_ref(a), want)
    assert np.array_equal(oracle.scan_f32_plain_f64(a), want)
    assert np.array_equal(oracle.abs_scan_f32(a), want)
    want_ex = np.concatenate([[0.0], want[:-1]])
    assert np.array_equal(oracle.scan_f32_ref(a, True), want_ex)


def test_f32_normal_compensated_vs_plain_double():
    n = 1 << 20
    a = synth.normal_f32(n, seed=0, stream=8)
    ref = oracle.scan_f32_ref(a)
    plain = oracle.scan_f32_plain_f64(a)
    den = oracle.abs_scan_f32(a)
    err, _ = oracle.max_rel_err(plain, ref, den)
    assert err < 1e-12


def test_f64_reference_exact_on_integers():
    n = 100_000
    a = synth.uniform_i64(n, 1 << 20, seed=9)
    assert np.array_equal(oracle.scan_f64_ref(a.astype(np.float64)),
                          np.cumsum(a).astype(np.float64))


# ---- segmented --------------------------------------------------------------

def random_offsets(n_seg, seed, max_len=40, empty_frac=0.2):
    lens = synth.uniform_i64(n_seg, max_len + 1, seed=seed, stream=1)
    drop = synth.unit_f32(n_seg, seed=seed, stream=2) < empty_frac
    lens = np.where(drop, 0, lens)
    return np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)


@pytest.mark.parametrize("excl", [False, True])
def test_segmented_is_per_segment_brute_force(excl):
    off = random_offsets(200, seed=4)
    n = int(off[-1])
    a = synth.raw_u64(n, seed=6).view(np.int64).astype(np.int32)
    y = oracle.seg_scan_i32(a, off, excl)
    for s in range(len(off) - 1):
        b, e = off[s], off[s + 1]
        assert y[b:e].tolist() == brute_scan(a[b:e].tolist(), excl, to_i32)


def test_segmented_special_cases():
    n = 10_000
    a = synth.uniform_i32(n, 16, seed=1)
    # one segment = plain scan
    assert np.array_equal(oracle.seg_scan_i32(a, [0, n]), oracle.scan_i32(a))
    # uniform segments = row-wise numpy cumsum
    rows, cols = 100, 100
    off = np.arange(rows + 1) * cols
    want = np.cumsum(a.reshape(rows, cols).astype(np.int64), axis=1).reshape(-1)
    assert np.array_equal(oracle.seg_scan_i32(a, off), want.astype(np.int32))
    # all segments of length 1: inclusive = a, exclusive = 0
    off1 = np.arange(n + 1)
    assert np.array_equal(oracle.seg_scan_i32(a, off1), a)
    assert np.array_equal(oracle.seg_scan_i32(a, off1, True), np.zeros(n, np.int32))
    # float segmented on the 2^-24 grid is exact
    f = synth.unit_f32(n, seed=2)
    kk = (f.astype(np.float64) * 2.0 ** 24).astype(np.int64)
    want_f = np.cumsum(kk.reshape(rows, cols), axis=1).reshape(-1) * 2.0 ** -24
    assert np.array_equal(oracle.seg_scan_f32_ref(f, off), want_f)
    # i64 segmented
    a64 = a.astype(np.int64)
    assert np.array_equal(oracle.seg_scan_i64(a64, off), want)


def test_segmented_rejects_bad_offsets():
    a = np.zeros(10, np.int32)
    for bad in ([0, 5], [1, 10], [0, 6, 4, 10]):
        with pytest.raises(ValueError):
            oracle.seg_scan_i32(a, bad)


# ---- reverse (suffix) scan: the gradient ------------------------------------

def test_suffix_ones_closed_form():
    rows, cols = 3, 1000
    g = np.ones((rows, cols), np.float32)
    i = np.arange(cols, dtype=np.float64)
    assert np.array_equal(oracle.rows_suffix_f32_ref(g), np.tile(cols - i, (rows, 1)))
    assert np.array_equal(oracle.rows_suffix_f32_ref(g, True), np.tile(cols - i - 1, (rows, 1)))


def test_suffix_is_jacobian_transpose_product():
    """Forward y_k = sum_{i<=k} a_i has Jacobian J[k, i] = [i <= k]; the
    gradient is J^T g (exclusive: J[k, i] = [i < k])."""
    cols = 64
    g = synth.normal_f32(2 * cols, seed=4).reshape(2, cols)
    J = np.tril(np.ones((cols, cols)))
    Jx = np.tril(np.ones((cols, cols)), -1)
    for r in range(2):
        gr = g[r].astype(np.float64)
        np.testing.assert_allclose(oracle.rows_suffix_f32_ref(g)[r], J.T @ gr,
                                   rtol=0, atol=1e-12)
        np.testing.assert_allclose(oracle.rows_suffix_f32_ref(g, True)[r], Jx.T @ gr,
                                   rtol=0, atol=1e-12)


def test_suffix_is_flip_scan_flip_exact_on_grid():
    rows, cols = 16, 4096
    g = synth.unit_f32(rows * cols, seed=5).reshape(rows, cols)
    k = (g.astype(np.float64) * 2.0 ** 24).astype(np.int64)
    want = np.flip(np.cumsum(np.flip(k, 1), 1), 1) * 2.0 ** -24
    assert np.array_equal(oracle.rows_suffix_f32_ref(g), want)
    assert np.array_equal(oracle.rows_suffix_abs_f32(g), want)
    g64 = g.astype(np.float64)
    assert np.array_equal(oracle.rows_suffix_f64_ref(g64), want)


# ---- the metric -------------------------------------------------------------

def test_metric_zero_denominator():
    y = np.array([0.0, 1.0, 2.0])
    ref = np.array([0.0, 1.0, 2.0])
    assert oracle.max_rel_err(y, ref, [0.0, 1.0, 2.0]) == (0.0, 0)
    err, k = oracle.max_rel_err([1e-30, 1.0, 2.0], ref, [0.0, 1.0, 2.0])
    assert err == math.inf and k == 0
    err, k = oracle.max_rel_err([0.0, 1.0, 2.5], ref, [0.0, 1.0, 4.0])
    assert err == pytest.approx(0.125) and k == 2


# ---- running maximum / minimum ------------------------------------------------

def _brute_running(a, op, exclusive):
    """O(n^2) definition: y_k = op over a[0..k] (exclusive: over a[0..k-1],
    the identity when empty), NaNs skipped as IEEE maxNum / minNum do."""
    if a.dtype == np.int32:
        ident = np.iinfo(np.int32).min if op == "max" else np.iinfo(np.int32).max
    else:
        ident = -np.inf if op == "max" else np.inf
    f = max if op == "max" else min
    out = []
    for k in range(a.size):
        part = [v for v in a[: k if exclusive else k + 1].tolist() if v == v]
        out.append(f(part) if part else ident)
    return np.array(out, dtype=a.dtype)


@pytest.mark.parametrize("op", ["max", "min"])
@pytest.mark.parametrize("exclusive", [False, True])
def test_running_max_min_brute_force(op, exclusive):
    for n in (1, 2, 7, 33, 64):
        a = (synth.uniform_i32(n, 1000, seed=n) - 500).astype(np.int32)
        assert np.array_equal(oracle.scan_op(a, op, exclusive), _brute_running(a, op, exclusive))
        f = synth.normal_f32(n, seed=n)
        f[::5] = np.nan  # maxNum / minNum skip NaNs
        assert np.array_equal(oracle.scan_op(f, op, exclusive), _brute_running(f, op, exclusive))


def test_running_max_min_closed_forms_and_invariants():
    k = np.arange(1000, dtype=np.int32)
    assert np.array_equal(oracle.scan_op(k, "max"), k)            # increasing: itself
    assert np.array_equal(oracle.scan_op(k[::-1].copy(), "max"), np.full(1000, 999, np.int32))
    assert np.array_equal(oracle.scan_op(k[::-1].copy(), "min"), k[::-1])
    assert oracle.scan_op(k, "max", True)[0] == np.iinfo(np.int32).min   # identity first
    assert oracle.scan_op(k, "min", True)[0] == np.iinfo(np.int32).max
    assert np.array_equal(oracle.scan_op(k, "max", True)[1:], k[:-1])   # exclusive = shift
    a = (synth.uniform_i32(50000, 1 << 20, seed=3) - (1 << 19)).astype(np.int32)
    y = oracle.scan_op(a, "max")
    assert np.all(np.diff(y.astype(np.int64)) >= 0) and y[-1] == a.max()
    assert np.all(np.isin(y, a))                    # every output is an input value
    z = oracle.scan_op(a, "min")
    assert np.all(np.diff(z.astype(np.int64)) <= 0) and z[-1] == a.min()
    f = synth.normal_f32(50000, seed=4)
    assert oracle.scan_op(f, "max")[-1] == f.max() and oracle.scan_op(f, "min")[-1] == f.min()
    assert oracle.scan_op(f, "max", True)[0] == -np.inf


# ---- stream compaction ----------------------------------------------------------

def test_compaction_definition():
    for n in (1, 5, 64, 1000):
        a = synth.uniform_i32(n, 1 << 20, seed=n)
        f = (synth.uniform_i32(n, 3, seed=n + 1)).astype(np.uint8)  # 0, 1, 2: nonzero keeps
        want = np.array([a[i] for i in range(n) if f[i] != 0], dtype=np.int32)
        got = oracle.compact(a, f)
        assert np.array_equal(got, want) and got.size == int(np.count_nonzero(f))
    x = synth.normal_f32(777, seed=2)
    assert np.array_equal(oracle.compact(x, np.ones(777, np.uint8)).view(np.uint32), x.view(np.uint32))
    assert oracle.compact(x, np.zeros(777, np.uint8)).size == 0
