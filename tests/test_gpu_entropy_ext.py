"""GPU parity of the entropy-side extensions against the oracle: the random-subsample estimate
(Sec. II.C) and the classical-noise subtraction (Sec. II.B). Bar as for qrng_minentropy."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12
FLOAT_KEYS = ("h_modify", "h_emp", "h_model", "d_u", "d_u_peak", "delta_fs", "delta_hm")


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a).view(np.uint8)).to("cuda")


def _same(got, want):
    for k in ("count", "max_count", "argmax", "bits"):
        assert got[k] == want[k], k
    for k in FLOAT_KEYS:
        assert abs(got[k] - want[k]) <= TOL, (k, got[k], want[k])
    for k in ("mean", "var"):
        assert abs(got[k] - want[k]) <= TOL * max(1.0, abs(want[k])), k


@pytest.mark.parametrize("fraction,sel_seed", [(1.0, 0), (0.5, 1), (0.05, 2024), (0.001, 7)])
@pytest.mark.parametrize("bits", [8, 12])
def test_sampled_estimate(qlib, gpu, oracle_mod, fraction, sel_seed, bits):
    s = W.adc_samples(2_000_003, 40 + bits, mu=(1 << bits) / 2, sigma=(1 << bits) / 16, bits=bits)
    got = qlib.qrng_minentropy_sampled(gpu, _dev(s).data_ptr(), s.size, bits, 1e-6, fraction, sel_seed)
    _same(got, oracle_mod.minentropy_sampled(s, bits, 1e-6, fraction, sel_seed))
    if fraction == 1.0:
        _same(got, oracle_mod.minentropy(s, bits, 1e-6))


def test_quantum_estimate(qlib, gpu, oracle_mod):
    on = W.adc_samples(1 << 22, 51, sigma=16.0)
    off = W.adc_samples(1 << 20, 52, sigma=6.0)
    got, hs = qlib.qrng_minentropy_quantum(gpu, _dev(on).data_ptr(), _dev(off).data_ptr(), on.size, off.size, 8, 1e-6)
    want, hs_want = oracle_mod.minentropy_quantum(on, off, 8, 1e-6)
    _same(got, want)
    assert abs(hs - hs_want) <= TOL
    assert got["h_model"] < oracle_mod.minentropy(on, 8, 1e-6)["h_model"]  # less noise, less entropy


def test_quantum_rejects_larger_classical_variance(qlib, gpu):
    on = W.adc_samples(10_000, 1, sigma=5.0)
    off = W.adc_samples(10_000, 2, sigma=9.0)
    with pytest.raises(qlib.QrngError) as e:
        qlib.qrng_minentropy_quantum(gpu, _dev(on).data_ptr(), _dev(off).data_ptr(), on.size, off.size, 8, 1e-6)
    assert e.value.status == qlib.QRNG_EINVAL


def test_sampled_bad_fraction(qlib, gpu):
    s = _dev(W.adc_samples(1000, 3))
    for f in (0.0, 1.5, -0.1):
        with pytest.raises(qlib.QrngError):
            qlib.qrng_minentropy_sampled(gpu, s.data_ptr(), 1000, 8, 1e-6, f, 1)
