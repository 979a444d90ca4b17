"""Plant plausible mistakes in a copy of the oracle and check that its pins
catch every one (CPU only).  The mutants are textual edits of oracle.c,
compiled into a temporary directory; the real oracle is untouched."""
import math
import os

import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")


def wide_range_f32(n, seed):
    """Normal floats scaled by 2^e, e uniform in [-40, 40]: their running sums
    need more than 53 bits, so double accumulation rounds."""
    e = synth.uniform_i32(n, 81, seed=seed, stream=5).astype(np.float64) - 40
    return (synth.normal_f32(n, seed=seed) * np.exp2(e)).astype(np.float32)


def meets_neumaier_bound(got, vals, excl):
    """|got_k - exact_k| <= 2u|exact_k| + O(n u^2) sum|a| (u = 2^-53), with
    exact_k from math.fsum (correctly rounded); plain double accumulation
    fails it on wide-range data."""
    vals = [float(v) for v in vals]
    exact = np.array([math.fsum(vals[:k + (0 if excl else 1)]) for k in range(len(vals))])
    den = np.cumsum(np.abs(vals))
    if excl:
        den = np.concatenate([[0.0], den[:-1]])
    bound = 2.0 ** -52 * np.abs(exact) + 2.0 ** -90 * den
    return bool(np.all(np.abs(np.asarray(got) - exact) <= bound))


def pins_pass(lib) -> bool:
    """A condensed run of the oracle's pins against `lib`."""
    g = read_golden("definition_example.txt")
    a = np.array(g["input"])
    checks = [
        oracle.scan_i32(a, lib=lib).tolist() == g["inclusive"],
        oracle.scan_i32(a, True, lib=lib).tolist() == g["exclusive"],
        oracle.scan_i64(a, lib=lib).tolist() == g["inclusive"],
        oracle.scan_i64(a, True, lib=lib).tolist() == g["exclusive"],
        oracle.scan_f32_ref(a, lib=lib).tolist() == g["inclusive"],
        oracle.scan_f32_ref(a, True, lib=lib).tolist() == g["exclusive"],
        oracle.rows_suffix_f32_ref(a.reshape(1, -1), lib=lib).ravel().tolist()
        == g["suffix_inclusive"],
        oracle.rows_suffix_f32_ref(a.reshape(1, -1), True, lib=lib).ravel().tolist()
        == g["suffix_exclusive"],
        oracle.seg_scan_i32(a, g["offsets"], lib=lib).tolist() == g["seg_inclusive"],
        oracle.seg_scan_i32(a, g["offsets"], True, lib=lib).tolist() == g["seg_exclusive"],
        oracle.seg_scan_f32_ref(a, g["offsets"], True, lib=lib).tolist() == g["seg_exclusive"],
        oracle.seg_scan_i64(a, g["offsets"], True, lib=lib).tolist() == g["seg_exclusive"],
    ]
    n = 4096
    k = (synth.unit_f32(n, seed=1).astype(np.float64) * 2 ** 24).astype(np.int64)
    f = (k * 2.0 ** -24).astype(np.float32)
    want = np.cumsum(k) * 2.0 ** -24
    checks += [
        np.array_equal(oracle.scan_f32_ref(f, lib=lib), want),
        np.array_equal(oracle.abs_scan_f32(-f, lib=lib), want),
        np.array_equal(oracle.abs_scan_f32(-f, True, lib=lib),
                       np.concatenate([[0.0], want[:-1]])),
        np.array_equal(oracle.rows_suffix_abs_f32(-f.reshape(1, -1), True, lib=lib).ravel(),
                       np.concatenate([np.flip(np.cumsum(np.flip(k)))[1:], [0]]) * 2.0 ** -24),
        np.array_equal(oracle.scan_f64_ref(f.astype(np.float64), lib=lib), want),
        np.array_equal(oracle.scan_f32_plain_f64(f, lib=lib), want),
        np.array_equal(oracle.rows_suffix_abs_f32(-f.reshape(1, -1), lib=lib).ravel(),
                       np.flip(np.cumsum(np.flip(k))) * 2.0 ** -24),
        np.array_equal(oracle.rows_suffix_f64_ref(f.reshape(2, -1).astype(np.float64),
                                                  lib=lib),
                       np.flip(np.cumsum(np.flip(k.reshape(2, -1), 1), 1), 1) * 2.0 ** -24),
        np.array_equal(oracle.rows_suffix_f32_ref(f.reshape(4, -1), lib=lib),
                       np.flip(np.cumsum(np.flip(k.reshape(4, -1), 1), 1), 1) * 2.0 ** -24),
        np.array_equal(oracle.scan_f32_plain_f64(f, True, lib=lib),
                       np.concatenate([[0.0], want[:-1]])),
        np.array_equal(oracle.scan_f64_ref(f.astype(np.float64), True, lib=lib),
                       np.concatenate([[0.0], want[:-1]])),
        np.array_equal(oracle.seg_abs_scan_f32(-f, [0, 100, n], lib=lib)[:100],
                       np.cumsum(k[:100]) * 2.0 ** -24),
    ]
    x = wide_range_f32(1500, seed=2)
    x64 = synth.normal_f64(1500, seed=2)
    for excl in (False, True):
        for got, vals in ((oracle.scan_f32_ref(x, excl, lib=lib), x.astype(np.float64)),
                          (oracle.scan_f64_ref(x64, excl, lib=lib), x64)):
            checks.append(meets_neumaier_bound(got, vals, excl))
    i = np.arange(1, 70001, dtype=np.int64)
    checks.append(oracle.reduce_i32(i.astype(np.int32), lib=lib)
                  == np.int64(i.sum() % (1 << 32)).astype(np.uint32).view(np.int32))
    checks.append(oracle.reduce_i64(i, lib=lib) == i.sum())
    # running max / min against their O(n^2) definition
    r = (synth.uniform_i32(40, 100, seed=6) - 50).astype(np.int32)
    rf = synth.normal_f32(40, seed=6)
    for op, f in (("max", max), ("min", min)):
        for excl in (False, True):
            for arr, ident in ((r, np.iinfo(np.int32).min if op == "max" else np.iinfo(np.int32).max),
                               (rf, -np.inf if op == "max" else np.inf)):
                want = [f(arr[: k if excl else k + 1].tolist()) if (k or not excl) else ident
                        for k in range(arr.size)]
                checks.append(np.array_equal(oracle.scan_op(arr, op, excl, lib=lib),
                                             np.array(want, dtype=arr.dtype)))
    # int64 and uint32 running max / min (their own identities and, for
    # uint32, unsigned order), against the same O(n^2) definition
    r64 = synth.uniform_i64(40, 1 << 32, seed=9).astype(np.int64) * 256 - (1 << 39)
    ru = (synth.uniform_i64(40, 1 << 32, seed=10)).astype(np.uint32)
    for op, f in (("max", max), ("min", min)):
        for excl in (False, True):
            for arr, ident in ((r64, np.iinfo(np.int64).min if op == "max" else np.iinfo(np.int64).max),
                               (ru, 0 if op == "max" else np.iinfo(np.uint32).max)):
                want = [f(arr[: k if excl else k + 1].tolist()) if (k or not excl) else ident
                        for k in range(arr.size)]
                checks.append(np.array_equal(oracle.scan_op(arr, op, excl, lib=lib),
                                             np.array(want, dtype=arr.dtype)))
    # uint32 sums: the modular running total (numpy uint32 cumsum wraps)
    for excl in (False, True):
        want = np.cumsum(ru, dtype=np.uint64) % (1 << 32)
        if excl:
            want = np.concatenate([[0], want[:-1]])
        checks.append(np.array_equal(oracle.scan_u32(ru, excl, lib=lib), want.astype(np.uint32)))
    # segmented max / min: each segment on its own (empty segments included)
    so = [0, 7, 7, 19, 40]
    for op, f in (("max", max), ("min", min)):
        for excl in (False, True):
            for arr, ident in ((r, np.iinfo(np.int32).min if op == "max" else np.iinfo(np.int32).max),
                               (rf, -np.inf if op == "max" else np.inf)):
                want = []
                for b, e in zip(so[:-1], so[1:]):
                    seg = arr[b:e].tolist()
                    want += [f(seg[: k if excl else k + 1]) if (k or not excl) else ident
                             for k in range(e - b)]
                checks.append(np.array_equal(oracle.seg_scan_op(arr, so, op, excl, lib=lib),
                                             np.array(want, dtype=arr.dtype)))
    cf = (synth.uniform_i32(50, 2, seed=7)).astype(np.uint8)
    cv = synth.uniform_i32(50, 1000, seed=8)
    checks.append(np.array_equal(oracle.compact(cv, cf, lib=lib),
                                 np.array([cv[i] for i in range(50) if cf[i]], np.int32)))
    return all(bool(c) for c in checks)


MUTANTS = {
    # (description): (original text, replacement text, occurrence index)
    "i32 exclusive adds before writing": (
        "            y[k] = (int32_t)run;\n            run += ak;",
        "            run += ak;\n            y[k] = (int32_t)run;", 0),
    "i64 dropped term": ("run += ak;", "run += ak & ~1ull;", 2),
    "i64 reduce off by one": ("for (int64_t k = 0; k < n; ++k) s += (uint64_t)a[k];",
                              "for (int64_t k = 1; k < n; ++k) s += (uint64_t)a[k];", 0),
    "reduce i32 wrong sign": ("s += (uint32_t)a[k];", "s -= (uint32_t)a[k];", 0),
    "neumaier wrong sign": ("acc->c += (acc->s - t) + x;", "acc->c -= (acc->s - t) + x;", 0),
    "neumaier lost error term": ("acc->c += (x - t) + acc->s;", "acc->c += (x - t);", 0),
    "f32 ref drops compensation in output": ("            y[k] = acc.s + acc.c;\n        }\n    }\n}\n\nvoid oracle_scan_f64_ref",
                                             "            y[k] = acc.s;\n        }\n    }\n}\n\nvoid oracle_scan_f64_ref", 0),
    "abs scan forgets fabs": ("neum_add(&acc, fabs((double)a[k]));\n        } else {",
                              "neum_add(&acc, ((double)a[k]));\n        } else {", 0),
    "segment bound off by one": ("if (e > b) oracle_scan_i32(a + b, y + b, e - b, exclusive);",
                                 "if (e > b) oracle_scan_i32(a + b, y + b, e - b - 1, exclusive);", 0),
    "segment uses next start": ("int64_t b = offsets[s], e = offsets[s + 1];\n        if (e > b) oracle_scan_f32_ref",
                                "int64_t b = offsets[s + 1], e = offsets[s + 1];\n        if (e > b) oracle_scan_f32_ref", 0),
    "suffix starts one early": ("for (int64_t i = cols - 1; i >= 0; --i) {", "for (int64_t i = cols - 2; i >= 0; --i) {", 0),
    "suffix f64 transposed index": ("const double* ar = a + r * cols;", "const double* ar = a + r;", 0),
    "max exclusive writes after the update": (
        "        if (exclusive) y[k] = run;\n        if (a[k] > run) run = a[k];",
        "        if (a[k] > run) run = a[k];\n        if (exclusive) y[k] = run;", 0),
    "min keeps the larger": ("if (a[k] < run) run = a[k];", "if (a[k] > run) run = a[k];", 0),
    "f32 max starts from +inf": ("float run = -INFINITY;", "float run = INFINITY;", 0),
    "f32 min uses fmaxf": ("run = fminf(run, a[k]);", "run = fmaxf(run, a[k]);", 0),
    "compaction keeps the dropped": ("if (flags[i] != 0) out[j++] = in[i];", "if (flags[i] == 0) out[j++] = in[i];", 0),
    "compaction writes in place of the input index": ("if (flags[i] != 0) out[j++] = in[i];",
                                                      "if (flags[i] != 0) { out[j] = in[j]; j++; }", 0),
    "i64 min starts from INT64_MIN": ("    int64_t run = INT64_MAX;", "    int64_t run = INT64_MIN;", 0),
    "u32 max compares signed": ("        if (a[k] > run) run = a[k];\n        if (!exclusive) y[k] = run;\n    }\n}\n\nvoid oracle_scan_min_u32",
                                "        if ((int32_t)a[k] > (int32_t)run) run = a[k];\n        if (!exclusive) y[k] = run;\n    }\n}\n\nvoid oracle_scan_min_u32", 0),
    "u32 min starts from 0": ("    uint32_t run = UINT32_MAX;", "    uint32_t run = 0;", 0),
    "u32 sum exclusive adds before writing": ("            y[k] = run;\n            run += a[k];",
                                              "            run += a[k];\n            y[k] = run;", 0),
    "segmented max does not restart": ("if (e > b) oracle_scan_max_i32(a + b, y + b, e - b, exclusive);",
                                       "if (e > b) oracle_scan_max_i32(a + offsets[0], y + offsets[0], e - offsets[0], exclusive);", 0),
    "segmented f32 min uses max": ("if (e > b) oracle_scan_min_f32(a + b, y + b, e - b, exclusive);",
                                   "if (e > b) oracle_scan_max_f32(a + b, y + b, e - b, exclusive);", 0),
    "plain double exclusive shifted": ("y[k] = run;\n            run += (double)a[k];",
                                       "run += (double)a[k];\n            y[k] = run;", 0),
}


def make_mutant(tmp_path, name, old, new, which):
    src = open(SRC).read()
    pos = -1
    for _ in range(which + 1):
        pos = src.find(old, pos + 1)
        assert pos >= 0, f"mutation site not found: {name}"
    mutated = src[:pos] + new + src[pos + len(old):]
    cpath = tmp_path / "mutant.c"
    cpath.write_text(mutated)
    so = oracle.build(force=True, src=str(cpath), out=str(tmp_path / "libmutant.so"))
    return oracle.load_library(so)


def test_real_oracle_passes_condensed_pins():
    assert pins_pass(None)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new, which = MUTANTS[name]
    lib = make_mutant(tmp_path, name, old, new, which)
    assert not pins_pass(lib), f"mutant survived: {name}"
