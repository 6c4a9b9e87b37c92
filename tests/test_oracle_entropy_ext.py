"""Pins for the oracle's entropy-side extensions: the random subsample of Sec. II.C (estimate the
corrected entropy from randomly selected samples) and the classical-noise subtraction of Sec. II.B
(quantum variance = laser-on variance - laser-off variance)."""
import json
import math
import os

import numpy as np
import pytest

from workloads import adc_samples

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL = 1e-12


def test_splitmix64_published_outputs(oracle_mod):
    with open(os.path.join(GOLDEN, "splitmix64_seed0.json")) as f:
        gold = json.load(f)
    for s, h in enumerate(gold["outputs_hex"], start=1):
        assert oracle_mod.splitmix64(gold["seed"], s) == int(h, 16)


def test_full_fraction_is_the_plain_estimate(oracle_mod):
    s = adc_samples(50_000, 3)
    a = oracle_mod.minentropy_sampled(s, 8, 1e-6, 1.0, 12345)
    b = oracle_mod.minentropy(s, 8, 1e-6)
    assert a == b


@pytest.mark.parametrize("fraction,seed", [(0.5, 1), (0.1, 7), (0.013, 99)])
def test_subsample_is_binomial_and_matches_selection(oracle_mod, fraction, seed):
    """The kept samples are the ones the generator selects (checked against the generator's own
    outputs) and their number is consistent with Binomial(N, fraction)."""
    s = adc_samples(20_000, 5 + seed)
    hist, bad = oracle_mod.histogram_sampled(s, 8, fraction, seed)
    thr = math.floor(fraction * 2.0 ** 53)
    keep = np.array([(oracle_mod.splitmix64(seed, i + 1) >> 11) < thr for i in range(s.size)])
    assert np.array_equal(hist, np.bincount(s[keep], minlength=256).astype(np.uint64))
    N, k = s.size, int(hist.sum())
    assert abs(k - fraction * N) < 6 * math.sqrt(N * fraction * (1 - fraction))


def test_subsample_widens_the_finite_size_term(oracle_mod):
    s = adc_samples(400_000, 11)
    full = oracle_mod.minentropy(s, 8, 1e-6)
    sub = oracle_mod.minentropy_sampled(s, 8, 1e-6, 0.25, 3)
    assert sub["count"] < full["count"]
    assert sub["delta_fs"] > full["delta_fs"] and sub["h_modify"] <= full["h_modify"] + 1e-9


def _sym_hist(center, sigma, scale=1e7):
    d = np.arange(256) - center
    h = np.rint(scale * np.exp(-(d.astype(np.float64) ** 2) / (2 * sigma * sigma))).astype(np.uint64)
    for k in range(1, min(center, 255 - center) + 1):
        h[center + k] = h[center - k]
    tail = 255 - center
    h[center + tail + 1:] = 0
    if center > tail:
        h[:center - tail] = 0
    return h


def _exact_var(h):
    v = np.arange(256)
    hh = [int(x) for x in h]
    N = sum(hh)
    s1 = sum(int(a) * b for a, b in zip(v, hh))
    s2 = sum(int(a) * int(a) * b for a, b in zip(v, hh))
    return (N * s2 - s1 * s1) / (N * N)


def _samples_from_hist(h):
    return np.repeat(np.arange(256, dtype=np.uint8), h.astype(np.int64))


def test_quantum_model_closed_form(oracle_mod):
    """Symmetric laser-on and laser-off histograms about integer codes: the quantum model is the
    Gaussian of variance var_on - var_off around the on mean, whose peak cell has mass
    erf(1 / (2 sqrt(2) sigma_q))."""
    on = _sym_hist(128, 20.0, scale=2e4)
    off = _sym_hist(90, 9.0, scale=2e4)
    rep, hsub = oracle_mod.minentropy_quantum(_samples_from_hist(on), _samples_from_hist(off), 8, 1e-6)
    var_q = _exact_var(on) - _exact_var(off)
    assert abs(rep["var"] - var_q) < 1e-9 * var_q
    peak = math.erf(1.0 / (2.0 * math.sqrt(2.0) * math.sqrt(var_q)))
    assert abs(rep["h_model"] - (-math.log2(peak))) < TOL
    full_on = oracle_mod.minentropy_from_hist(on, 8, 1e-6)
    full_off = oracle_mod.minentropy_from_hist(off, 8, 1e-6)
    assert abs(hsub - (full_on["h_model"] - full_off["h_model"])) < TOL
    assert rep["delta_hm"] == full_on["delta_hm"] and rep["d_u"] == full_on["d_u"]
    assert abs(rep["h_modify"] - max(0.0, rep["h_model"] - rep["delta_hm"])) < TOL


def test_quantum_without_classical_noise_is_the_plain_estimate(oracle_mod):
    """A laser-off stream with no spread (zero classical variance) leaves the model unchanged."""
    on = adc_samples(100_000, 21)
    off = np.full(5000, 128, dtype=np.uint8)
    rep, hsub = oracle_mod.minentropy_quantum(on, off, 8, 1e-6)
    plain = oracle_mod.minentropy(on, 8, 1e-6)
    for k in ("h_model", "h_modify", "var", "d_u", "delta_hm"):
        assert abs(rep[k] - plain[k]) < TOL, k
    assert abs(hsub - plain["h_model"]) < TOL


def test_quantum_rejects_classical_variance_above_total(oracle_mod):
    on = adc_samples(20_000, 1, sigma=5.0)
    off = adc_samples(20_000, 2, sigma=9.0)
    with pytest.raises(ValueError):
        oracle_mod.minentropy_quantum(on, off, 8, 1e-6)
