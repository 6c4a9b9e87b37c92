"""The oracle pins must catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (in a temporary directory, on
the CPU), builds it, and runs the pin tests against the planted copy: at least one pin has to
fail. The committed oracle is never modified.
"""
import importlib.util
import os
import shutil

import numpy as np
import pytest

import test_oracle_entropy as E
import test_oracle_entropy_ext as X
import test_oracle_toeplitz as T

ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")

MUTANTS = {
    # extraction
    "transposed_seed_index": ("a[n - 1 + i - j] & r[j]", "a[i + j] & r[j]"),
    "dropped_last_column": ("for (uint64_t j = 0; j < n; ++j) sum +=", "for (uint64_t j = 0; j + 1 < n; ++j) sum +="),
    "modified_identity_off_by_one": ("sum += r[n - m + i];", "sum += r[n - m + i - 1];"),
    "modified_seed_mirrored": ("a[n - m - 1 + i - j] & r[j]", "a[i + j] & r[j]"),
    "msb_first_bit_order": ("return (buf[t >> 3] >> (t & 7)) & 1;", "return (buf[t >> 3] >> (7 - (t & 7))) & 1;"),
    # entropy
    "half_cell_shift": ("((double)v - 0.5 - mu) / sigma;", "((double)v - mu) / sigma;"),
    "lower_tail_dropped": ("double lo = (v == 0) ? -INFINITY :", "double lo = (v == 0) ? (-0.5 - mu) / sigma :"),
    "central_cell_sign": ("return 0.5 * (erf(z * r) - erf(y * r));", "return 0.5 * (erf(z * r) + erf(y * r));"),
    "sample_variance": ("double var = (double)num / ((double)N * (double)N);",
                        "double var = (double)num / ((double)N * (double)(N - 1));"),
    "distance_missing_half": ("rep->d_u = 0.5 * d;", "rep->d_u = d;"),
    "correction_wrong_power": ("ldexp(1.0, -bits - 1)", "ldexp(1.0, -bits)"),
    "finite_size_term_dropped": ("rep->delta_hm = log2((rep->d_u + rep->delta_fs)",
                                 "rep->delta_hm = log2((rep->d_u)"),
    "peak_distance_at_model_peak": ("rep->d_u_peak = 0.5 * fabs((double)maxc / (double)N - P[argmax]);",
                                    "rep->d_u_peak = 0.5 * fabs((double)maxc / (double)N - pmax);"),
    "peak_distance_missing_half": ("rep->d_u_peak = 0.5 * fabs(", "rep->d_u_peak = 1.0 * fabs("),
    "argmax_highest_code_on_ties": ("if (hist[v] > maxc) { maxc = hist[v];", "if (hist[v] >= maxc) { maxc = hist[v];"),
    "finite_size_without_code_count": ("2.0 * ((double)K * log(2.0) + log(1.0 / eps))", "2.0 * (log(1.0 / eps))"),
    "finite_size_without_confidence": ("2.0 * ((double)K * log(2.0) + log(1.0 / eps))", "2.0 * ((double)K * log(2.0))"),
    "finite_size_bits_for_codes": ("2.0 * ((double)K * log(2.0) + log(1.0 / eps))",
                                   "2.0 * ((double)bits * log(2.0) + log(1.0 / eps))"),
    # entropy-side extensions
    "quantum_variance_added": ("double var_q = rep->var - off.var;", "double var_q = rep->var + off.var;"),
    "subsample_wrong_bits": (">> 11) >= thr) continue;", ">> 10) >= thr) continue;"),
    "splitmix_wrong_shift": ("z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;", "z = (z ^ (z >> 28)) * 0x94D049BB133111EBull;"),
}

PINS = [
    (T.test_standard_equals_polynomial_product, dict(n=97, m=50)),
    (T.test_standard_equals_paper_circulant_route, dict(n=129, m=100)),
    (T.test_modified_equals_paper_circulant_route, dict(n=255, m=200)),
    (T.test_modified_identity_block, dict(n=64, m=32)),
    (T.test_standard_columns_are_seed_windows_with_equal_diagonals, dict(n=16, m=8)),
    (E.test_integer_mean_peak_closed_form, dict(center=100, sigma=7.5)),
    (E.test_one_bit_source_closed_form, dict(h0=123456, h1=654321)),
    (E.test_reflection_invariance, dict(seed=2)),
    (E.test_flat_histogram_has_bits_of_entropy, dict(bits=8)),
    (E.test_peak_distance_closed_form, dict()),
    (E.test_argmax_lowest_code_on_ties, dict()),
    (E.test_finite_size_term_covers_multinomial_deviation, dict(bits=4, N=400, eps=0.05)),
    (X.test_splitmix64_published_outputs, dict()),
    (X.test_quantum_model_closed_form, dict()),
    (X.test_subsample_is_binomial_and_matches_selection, dict(fraction=0.5, seed=1)),
]


def _planted_oracle(tmp_path, name, old, new):
    d = tmp_path / name
    d.mkdir()
    src = open(os.path.join(ORACLE_DIR, "qrng_oracle.c")).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    (d / "qrng_oracle.c").write_text(src.replace(old, new))
    shutil.copy(os.path.join(ORACLE_DIR, "__init__.py"), d / "__init__.py")
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{name}", d / "__init__.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    mod = _planted_oracle(tmp_path, name, old, new)
    failures = []
    for fn, kw in PINS:
        try:
            fn(mod, **kw)
        except (AssertionError, ValueError) as e:  # a pin failed: the mistake is caught
            failures.append(fn.__name__)
    assert failures, f"no pin caught the planted mistake {name!r}"


def test_unplanted_copy_passes_every_pin(tmp_path):
    mod = _planted_oracle(tmp_path, "none", "#define ORACLE_OK 0", "#define ORACLE_OK 0")
    for fn, kw in PINS:
        fn(mod, **kw)
