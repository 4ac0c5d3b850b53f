"""Plants plausible mistakes in the C oracle (on the CPU) and checks that the
pins of test_oracle_pins.py catch each one.

Every mutant is a one-token edit of ``oracle/composite_oracle.c`` compiled to
its own shared object; the pins then run against it in place of the real
oracle.  A mutant that no pin rejects would mean the pins cannot tell that
mistake from the definition.
"""
import ctypes
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "composite_oracle.c")

MUTANTS = {
    "drops_first_member": ("for (m = 0; m < n; ++m) {\n        const uint8_t",
                           "for (m = 1; m < n; ++m) {\n        const uint8_t"),
    "transposed_pixel_index": ("counts[y * width + x] += sign", "counts[x * height + y] += sign"),
    "counts_only_value_one": ("if (row[x] != 0)", "if (row[x] == 1)"),
    "ignores_row_pitch": ("const uint8_t *row = member + y * row_pitch;",
                          "const uint8_t *row = member + y * width;"),
    "remove_adds": ("counts[y * width + x] += sign", "counts[y * width + x] += 1"),
    "bucket_rounds_to_nearest": ("(255 * (uint64_t)counts[p]) / (uint64_t)n_members",
                                 "(255 * (uint64_t)counts[p] + (uint64_t)n_members / 2) / (uint64_t)n_members"),
    "bucket_scale_256": ("(255 * (uint64_t)counts[p])", "(256 * (uint64_t)counts[p])"),
    "lut_green_reversed": ("lut[4 * b + 1] = (uint8_t)(255 - b);", "lut[4 * b + 1] = (uint8_t)(b);"),
    "rgba_channel_swap": ("rgba[4 * p + c] = lut[4 * (int64_t)bucket[p] + c];",
                          "rgba[4 * p + c] = lut[4 * (int64_t)bucket[p] + (3 - c)];"),
    "mean_divides_by_n_minus_1": ("sums[p] / (double)n_members", "sums[p] / (double)(n_members - 1 + (n_members == 1))"),
    "depth_drops_sign": ("sums[y * width + x] += (double)sign * (double)row[x];",
                         "sums[y * width + x] += (double)row[x];"),
    "histogram_skips_class_zero": ("        hist[bucket[p]] += 1;", "        hist[bucket[p]] += bucket[p] != 0;"),
}

PINS = [
    lambda: pins.test_count_matches_nested_threshold_identity(1, 64, 48, 7),
    lambda: pins.test_count_matches_nested_threshold_identity(11, 257, 131, 37),
    lambda: pins.test_count_range_and_sum_invariants(2),
    pins.test_count_order_independent,
    pins.test_single_member_is_its_own_mask,
    pins.test_closed_forms,
    pins.test_nonzero_bytes_count_once,
    pins.test_strided_members_read_correctly,
    pins.test_add_then_remove_equals_recompute,
    pins.test_remove_of_unadded_member_is_underflow,
    pins.test_bucket_large_counts_and_zero_members,
    pins.test_default_lut_is_white_to_saturated_blue,
    pins.test_rgba_is_a_table_lookup,
    pins.test_mean_depth_against_exact_rationals,
    pins.test_mean_depth_special_cases,
    pins.test_mean_depth_add_then_remove,
    pins.test_histogram_counts_every_pixel_once,
    pins.test_histogram_closed_forms,
    pins.test_brute_force_on_random_8x8_inputs,
]


def _bucket_pin_small():
    # the exhaustive floor characterisation, over N <= 64 to stay quick
    import numpy as np
    for n in range(1, 65):
        c = np.arange(n + 1, dtype=np.int64)
        b = oracle.bucket(c, n).astype(np.int64)
        assert np.all(b * n <= 255 * c) and np.all(255 * c < (b + 1) * n)


PINS.append(_bucket_pin_small)


def _mutant_lib(tmp_path, name):
    src = open(SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.run(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-o", str(so), str(path)], check=True)
    return so


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(tmp_path, name, monkeypatch):
    so = _mutant_lib(tmp_path, name)
    real = oracle._load()
    mutant = ctypes.CDLL(str(so))
    for fn in ("oracle_count_apply", "oracle_bucket", "oracle_rgba", "oracle_default_lut",
               "oracle_depth_apply", "oracle_mean", "oracle_histogram"):
        getattr(mutant, fn).restype = getattr(real, fn).restype
        getattr(mutant, fn).argtypes = getattr(real, fn).argtypes
    monkeypatch.setattr(oracle, "_lib", mutant)
    failed = []
    for pin in PINS:
        try:
            pin()
        except (AssertionError, ValueError):
            failed.append(pin)
    assert failed, f"no pin rejects the mutant {name}"


def test_unmutated_oracle_passes_every_pin():
    for pin in PINS:
        pin()
