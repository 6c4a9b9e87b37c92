"""Pins for the oracle's min-entropy estimate (Sec. II) and output length (Sec. III.B).

Expected values come from closed forms and special cases, not from the oracle's formula:
  * flat and point-mass histograms (H_min = bits and 0, Sec. II.A definition);
  * a symmetric histogram with an integer mean, whose model peak bin has mass erf(1/(2 sqrt(2) sigma));
  * a 1-bit source, where the model has two cells that split at 1/2 (standard normal CDF from
    scipy) and every quantity has a closed form;
  * reflection and shift invariance of the Gaussian model (catches a half-cell offset or a tail
    put in the wrong end code);
  * the histogram equals numpy's bincount;
  * the distance over U = {argmax P'} (Sec. II.C) on a histogram whose empirical peak is not the
    model's peak, and the lowest-code rule for equal peaks;
  * the finite-size term: multinomial draws from a known distribution stay within it at least
    a 1 - eps fraction of the time, and it is where Weissman's L1 tail bound reaches eps;
  * the worked example of Sec. II.B (loose pin, values in tests/golden/).
"""
import json
import math
import os

import numpy as np
import pytest

from workloads import adc_quantise, adc_samples, attack_voltages

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL = 1e-12


def _flat_hist(bits, per_code):
    return np.full(1 << bits, per_code, dtype=np.uint64)


@pytest.mark.parametrize("bits", [1, 2, 5, 8, 12, 16])
def test_flat_histogram_has_bits_of_entropy(oracle_mod, bits):
    rep = oracle_mod.minentropy_from_hist(_flat_hist(bits, 3), bits, 1e-6)
    assert abs(rep["h_emp"] - bits) < TOL
    assert rep["count"] == 3 << bits


def test_flat_samples_through_histogram(oracle_mod):
    s = np.tile(np.arange(256, dtype=np.uint8), 40)
    rep = oracle_mod.minentropy(s, 8, 1e-6)
    assert abs(rep["h_emp"] - 8.0) < TOL
    assert abs(rep["mean"] - 127.5) < TOL


@pytest.mark.parametrize("bits,code", [(8, 0), (8, 200), (8, 255), (3, 5)])
def test_point_mass_has_zero_entropy(oracle_mod, bits, code):
    h = np.zeros(1 << bits, dtype=np.uint64)
    h[code] = 1000
    rep = oracle_mod.minentropy_from_hist(h, bits, 1e-6)
    assert rep["h_emp"] == 0.0 and rep["var"] == 0.0 and rep["h_model"] == 0.0
    assert rep["d_u"] == 0.0 and rep["h_modify"] == 0.0
    assert rep["argmax"] == code


def _symmetric_gaussian_hist(center, sigma, scale=1e7, bits=8):
    d = np.arange(-center, (1 << bits) - center)
    h = np.rint(scale * np.exp(-(d.astype(np.float64) ** 2) / (2 * sigma * sigma))).astype(np.uint64)
    # force exact symmetry about `center`
    for k in range(1, min(center, (1 << bits) - 1 - center) + 1):
        h[center + k] = h[center - k]
    return h


@pytest.mark.parametrize("center,sigma", [(128, 16.0), (100, 7.5), (60, 3.0)])
def test_integer_mean_peak_closed_form(oracle_mod, center, sigma):
    """Symmetric histogram about an integer code c: the model mean is exactly c, and the model
    peak cell [c-1/2, c+1/2] has mass Phi(1/(2s)) - Phi(-1/(2s)) = erf(1/(2 sqrt(2) s)), with s
    the population standard deviation of the histogram (computed here with exact integers)."""
    h = _symmetric_gaussian_hist(center, sigma)
    tail = (1 << 8) - 1 - center
    h[center + tail + 1:] = 0
    if center > tail:
        h[:center - tail] = 0
    v = np.arange(256, dtype=object)
    hh = [int(x) for x in h]
    N = sum(hh)
    s1 = sum(int(a) * b for a, b in zip(v, hh))
    s2 = sum(int(a) * int(a) * b for a, b in zip(v, hh))
    assert s1 == center * N
    var = (N * s2 - s1 * s1) / (N * N)
    rep = oracle_mod.minentropy_from_hist(h, 8, 1e-6)
    assert abs(rep["mean"] - center) < TOL
    assert abs(rep["var"] - var) < 1e-9 * var
    peak = math.erf(1.0 / (2.0 * math.sqrt(2.0) * math.sqrt(var)))
    assert abs(rep["h_model"] - (-math.log2(peak))) < TOL


@pytest.mark.parametrize("h0,h1", [(500, 500), (123456, 654321), (7, 1), (1, 999)])
def test_one_bit_source_closed_form(oracle_mod, h0, h1):
    """K = 2 codes: mean mu = h1/N, variance mu(1-mu); the model puts Phi((1/2-mu)/sigma) in code
    0 and the rest in code 1, so d_U = |p'_0 - P_0| and every later quantity is a closed form."""
    from scipy.stats import norm

    N = h0 + h1
    mu = h1 / N
    sigma = math.sqrt(mu * (1 - mu))
    p0 = float(norm.cdf((0.5 - mu) / sigma))
    eps = 1e-6
    rep = oracle_mod.minentropy_from_hist(np.array([h0, h1], dtype=np.uint64), 1, eps)
    assert abs(rep["h_model"] - (-math.log2(max(p0, 1 - p0)))) < TOL
    assert abs(rep["d_u"] - abs(h0 / N - p0)) < TOL
    delta = 0.5 * math.sqrt(2.0 * (2 * math.log(2.0) + math.log(1 / eps)) / N)
    assert abs(rep["delta_fs"] - delta) < TOL
    dhm = math.log2((rep["d_u"] + delta) * 4.0 + 1.0)
    assert abs(rep["delta_hm"] - dhm) < TOL
    assert abs(rep["h_modify"] - max(0.0, rep["h_model"] - dhm)) < TOL
    if h0 == h1:
        assert abs(rep["h_model"] - 1.0) < TOL and rep["d_u"] < TOL


def _model_cell(hist, code):
    """Mass of code `code` under the Gaussian with the histogram's mean and population variance
    (exact integer moments), the cell [code - 1/2, code + 1/2] (scipy's normal CDF)."""
    from scipy.stats import norm

    hh = [int(x) for x in hist]
    N = sum(hh)
    s1 = sum(v * c for v, c in enumerate(hh))
    s2 = sum(v * v * c for v, c in enumerate(hh))
    mu = s1 / N
    sigma = math.sqrt((N * s2 - s1 * s1) / (N * N))
    return float(norm.cdf((code + 0.5 - mu) / sigma) - norm.cdf((code - 0.5 - mu) / sigma))


def test_peak_distance_closed_form(oracle_mod):
    """Sec. II.C restricted to U = {argmax P'}: d = |P'(x*) - P(x*)| / 2 at the empirical peak x*.
    Here the measured peak (code 2, 40 %) is not the model's (the mean is 2.95, so code 3), so a
    distance taken at the model's peak, or without the 1/2, differs."""
    h = np.zeros(8, dtype=np.uint64)
    h[2], h[3], h[4] = 40, 25, 35
    rep = oracle_mod.minentropy_from_hist(h, 3, 1e-6)
    assert rep["argmax"] == 2 and rep["max_count"] == 40
    assert abs(rep["mean"] - 2.95) < TOL
    p2, p3 = _model_cell(h, 2), _model_cell(h, 3)
    assert p3 > p2  # the model's own peak sits elsewhere
    assert abs(rep["h_model"] - (-math.log2(p3))) < TOL
    assert abs(rep["d_u_peak"] - 0.5 * abs(0.40 - p2)) < TOL


def test_argmax_lowest_code_on_ties(oracle_mod):
    """Two codes share the largest count: H_min does not depend on which is reported, and the
    report takes the lower code, so d over U = {argmax P'} is taken there."""
    h = np.zeros(8, dtype=np.uint64)
    h[1], h[2], h[3], h[5] = 30, 15, 30, 25
    rep = oracle_mod.minentropy_from_hist(h, 3, 1e-6)
    assert rep["argmax"] == 1 and rep["max_count"] == 30
    assert abs(rep["h_emp"] - (-math.log2(0.30))) < TOL
    p1, p3 = _model_cell(h, 1), _model_cell(h, 3)
    assert abs(p1 - p3) > 1e-3  # an asymmetric histogram: the two ties have different model cells
    assert abs(rep["d_u_peak"] - 0.5 * abs(0.30 - p1)) < TOL


@pytest.mark.parametrize("bits,N,eps", [(4, 400, 0.05), (3, 2000, 0.1)])
def test_finite_size_term_covers_multinomial_deviation(oracle_mod, bits, N, eps):
    """The finite-size term is read as a confidence bound on the statistical distance between
    the empirical distribution of N samples and the true one. Drawn N samples at a time from a
    known distribution, the distance exceeds it in at most an eps fraction of the draws; and it is
    the deviation at which Weissman et al.'s tail bound P(||p^ - p||_1 >= t) <= (2^K - 2)
    exp(-N t^2 / 2) (K codes, t = twice the statistical distance) comes down to eps, up to
    replacing 2^K - 2 by 2^K."""
    K = 1 << bits
    g = np.random.Generator(np.random.PCG64(17 + bits))
    p = g.uniform(0.5, 1.5, K)
    p /= p.sum()
    draws = g.multinomial(N, p, size=6000)
    tv = 0.5 * np.abs(draws / N - p).sum(axis=1)
    h = np.zeros(K, dtype=np.uint64)
    h[0] = N  # delta depends on N, K and eps only
    delta = oracle_mod.minentropy_from_hist(h, bits, eps)["delta_fs"]
    assert np.mean(tv > delta) <= eps
    assert np.mean(tv > 0.5 * delta) > eps  # and it is not vacuous by a factor of two
    tail = (2.0 ** K - 2) * math.exp(-N * (2 * delta) ** 2 / 2)
    assert tail <= eps * (1 + 1e-12)
    assert tail >= eps * (2.0 ** K - 2) / 2.0 ** K * (1 - 1e-12)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_reflection_invariance(oracle_mod, seed):
    """Reversing the code order (v -> K-1-v) mirrors the Gaussian model about the mean, so the
    model entropy and the distance do not change."""
    s = adc_samples(200000, seed, mu=90.0 + 20 * seed, sigma=5.0 + 4 * seed)
    h, _ = oracle_mod.histogram(s, 8)
    a = oracle_mod.minentropy_from_hist(h, 8, 1e-6)
    b = oracle_mod.minentropy_from_hist(h[::-1].copy(), 8, 1e-6)
    for key in ("h_emp", "h_model", "d_u", "var", "delta_hm", "h_modify"):
        assert abs(a[key] - b[key]) < 1e-11, key
    assert abs(a["mean"] + b["mean"] - 255.0) < 1e-11


def test_shift_invariance(oracle_mod):
    """Moving every sample by the same number of codes, far from the end codes, leaves the model
    entropy and the distance unchanged."""
    s = adc_samples(100000, 8, mu=100.0, sigma=6.0)
    h, _ = oracle_mod.histogram(s, 8)
    a = oracle_mod.minentropy_from_hist(h, 8, 1e-6)
    b = oracle_mod.minentropy_from_hist(np.roll(h, 37), 8, 1e-6)
    for key in ("h_emp", "h_model", "d_u", "var"):
        assert abs(a[key] - b[key]) < 1e-11, key
    assert abs(b["mean"] - a["mean"] - 37) < 1e-11


@pytest.mark.parametrize("bits", [4, 8, 11, 16])
def test_histogram_is_bincount(oracle_mod, bits):
    g = np.random.Generator(np.random.PCG64(bits))
    dt = np.uint8 if bits <= 8 else np.uint16
    s = g.integers(0, 1 << bits, 50000).astype(dt)
    h, bad = oracle_mod.histogram(s, bits)
    assert bad == 0
    assert np.array_equal(h, np.bincount(s, minlength=1 << bits).astype(np.uint64))
    if bits < 8:
        s2 = s.copy()
        s2[10] = 1 << bits
        assert oracle_mod.histogram(s2, bits)[1] == 1
        with pytest.raises(ValueError):
            oracle_mod.minentropy(s2, bits, 1e-6)


def test_correction_monotone_and_finite_size(oracle_mod):
    """Delta H_m grows with the distance and with 1/eps, and shrinks with the sample count."""
    s = adc_samples(1 << 20, 4)
    h, _ = oracle_mod.histogram(s, 8)
    r1 = oracle_mod.minentropy_from_hist(h, 8, 1e-3)
    r2 = oracle_mod.minentropy_from_hist(h, 8, 1e-9)
    assert r2["delta_fs"] > r1["delta_fs"] and r2["delta_hm"] > r1["delta_hm"]
    r4 = oracle_mod.minentropy_from_hist(h * np.uint64(4), 8, 1e-3)
    assert abs(r4["delta_fs"] - r1["delta_fs"] / 2) < 1e-15
    assert abs(r4["d_u"] - r1["d_u"]) < 1e-15
    # a distorted histogram (one code inflated) is further from the model
    h2 = h.copy()
    h2[128] += 20000
    r3 = oracle_mod.minentropy_from_hist(h2, 8, 1e-3)
    assert r3["d_u"] > r1["d_u"] and r3["delta_hm"] > r1["delta_hm"]
    assert 0 <= r1["h_modify"] <= r1["h_model"]


def test_worked_example_sec2b_loose(oracle_mod):
    """Sec. II.B: 5-bit sampling of V and of the attacked V' on [-5, 5] gives H(V) ~ 2.99 and
    H'(V') ~ 2.94, so the attack leaks I(G:E) = H(V) - H'(V') > 0. Loose pin: the paper does not
    say how its ADC rounds, so the stated values are matched to within the golden tolerance."""
    with open(os.path.join(GOLDEN, "worked_example_sec2b.json")) as f:
        gold = json.load(f)
    v, v_att = attack_voltages(gold["samples"], gold["rng_seed"])
    hv = oracle_mod.minentropy(adc_quantise(v, 5, -5.0, 5.0), 5, 1e-6)["h_emp"]
    hva = oracle_mod.minentropy(adc_quantise(v_att, 5, -5.0, 5.0), 5, 1e-6)["h_emp"]
    assert abs(hv - gold["H_V"]) <= gold["tol"]
    assert abs(hva - gold["H_V_attacked"]) <= gold["tol"]
    assert hv > hva


@pytest.mark.parametrize("n,h,bits,eps,want", [
    (1024, 8.0, 8, 2.0 ** -10, 1004),   # 1024 - 2*10
    (4096, 4.0, 8, 1.0, 2048),          # no security term
    (1000, 3.3, 5, 0.5, 658),           # floor(660 - 2)
    (100, 0.1, 8, 1e-6, 0),             # negative -> 0
])
def test_output_length(oracle_mod, n, h, bits, eps, want):
    assert oracle_mod.output_length(n, h, bits, eps) == want
