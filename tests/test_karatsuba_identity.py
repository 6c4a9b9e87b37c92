"""The block-Karatsuba identity the GEMM_KARATSUBA route relies on, checked on the CPU against the
oracle's Toeplitz hash (Sec. III.B standard, Sec. III.D modified) with plain numpy bit matrices.

Zero-pad the m x n_t Toeplitz matrix T[i][j] = a[n_t - 1 + i - j] to multiples of span = h 2^L
and cut it into h x h blocks; a 2 x 2 group [[T_d, T_d+1], [T_d-1, T_d]] times (x0, x1) is, over
GF(2), (T_d (x0^x1) ^ (T_d+1 ^ T_d) x1, T_d (x0^x1) ^ (T_d-1 ^ T_d) x0). After L rounds the
3^L sub-products z = (z_1 .. z_L) (0 = A, 1 = B, 2 = C) read seeds a_z (a XOR-shifted by +-h 2^(l-1)
per B/C digit) on every span-th h-block, and inputs XOR-ed over the raw h-blocks whose level bits
the digits allow; output h-block 2^L R + q is the XOR of the 2^L sub-products that q selects.
This module restates that on matrices (not the kernels' word arithmetic), so that a wrong shift
sign, digit order or selection rule fails against the definition.
"""
import numpy as np
import pytest

import workloads as W

STD, MOD = 0, 1


def _bits(buf, nbits):
    return np.unpackbits(np.asarray(buf, dtype=np.uint8), bitorder="little")[:nbits].astype(np.int64)


def _karatsuba_hash(a, x, n_t, m, L, h, b_shift=-1):
    """Toeplitz part of the hash of one block via L levels of 2 x 2 block splits (b_shift: the sign
    of a B digit's seed shift in t; C takes the other)."""
    span = h << L
    R = -(-m // span)
    C = -(-n_t // span)
    M, K = R * span, C * span
    xp = np.zeros(K, dtype=np.int64)
    xp[:n_t] = x[:n_t]

    def a_at(t):  # zero-extended seed
        t = np.asarray(t)
        out = np.zeros(t.shape, dtype=np.int64)
        ok = (t >= 0) & (t < a.size)
        out[ok] = a[t[ok]]
        return out

    G = 3 ** L
    y = np.zeros(M, dtype=np.int64)
    qpar = {}
    for z in range(G):
        digits = [(z // 3 ** l) % 3 for l in range(L)]
        # derived seed: a_z(t) = XOR over the chosen shifts of a(t + shift); a B digit at level l
        # pairs T_d+1 (seed shifted by -h 2^(l-1) in t) with T_d, a C digit T_d-1 (shift +)
        shifts = [0]
        for l, d in enumerate(digits):
            s = h << l
            if d == 1:
                shifts = shifts + [sh + b_shift * s for sh in shifts]
            elif d == 2:
                shifts = shifts + [sh - b_shift * s for sh in shifts]

        def a_z(t):
            v = np.zeros(np.asarray(t).shape, dtype=np.int64)
            for sh in shifts:
                v ^= a_at(np.asarray(t) + sh)
            return v

        # sub-product rows: every span-th h-block of rows, columns likewise (virtual coordinates)
        rows = np.concatenate([r * span + np.arange(h) for r in range(R)])
        cols = np.concatenate([c * span + np.arange(h) for c in range(C)])
        Tz = a_z(n_t - 1 + rows[:, None] - cols[None, :])
        # derived input: XOR of the raw h-blocks 2^L c + q over the q the digits allow
        qs = [q for q in range(1 << L)
              if all(d == 0 or (d == 1 and (q >> l) & 1) or (d == 2 and not (q >> l) & 1)
                     for l, d in enumerate(digits))]
        xz = np.zeros(C * h, dtype=np.int64)
        for c in range(C):
            for q in qs:
                xz[c * h:(c + 1) * h] ^= xp[(c * (1 << L) + q) * h:(c * (1 << L) + q + 1) * h]
        qpar[z] = (Tz @ xz) & 1
    for r in range(R):
        for q in range(1 << L):
            acc = np.zeros(h, dtype=np.int64)
            for sset in range(1 << L):  # subsets of the levels whose digit is B or C
                z = sum(((1 + ((q >> l) & 1)) if (sset >> l) & 1 else 0) * 3 ** l for l in range(L))
                acc ^= qpar[z][r * h:(r + 1) * h]
            y[((r << L) + q) * h:((r << L) + q + 1) * h] = acc
    return y[:m]


@pytest.mark.parametrize("L,h", [(1, 4), (2, 4), (3, 4), (1, 8), (2, 16), (3, 8), (2, 32), (4, 4), (4, 8)])
@pytest.mark.parametrize("n,m,form", [(300, 170, STD), (300, 170, MOD), (257, 257, STD), (129, 40, MOD),
                                      (64, 63, MOD), (1, 1, STD)])
def test_block_karatsuba_equals_definition(oracle_mod, L, h, n, m, form):
    seed = W.random_bits(n + m - 1 if form == STD else n - 1, 11 * n + m + L)
    raw = W.random_bits(n, 7 * n + m + h)
    want = np.unpackbits(oracle_mod.toeplitz(raw, n, m, seed, form), bitorder="little")[:m]
    n_t = n - m if form == MOD else n
    a = _bits(seed, n_t + m - 1)
    x = _bits(raw, n)
    y = _karatsuba_hash(a, x, n_t, m, L, h)
    if form == MOD:
        y ^= x[n - m:n]
    assert np.array_equal(y, want)


@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_a_wrong_shift_sign_is_caught(oracle_mod, L):
    """The identity test is sensitive to the seed-shift direction: B and C shifts swapped fail."""
    n, m = 300, 170
    seed = W.random_bits(n + m - 1, 3 + L)
    raw = W.random_bits(n, 4 + L)
    want = np.unpackbits(oracle_mod.toeplitz(raw, n, m, seed, STD), bitorder="little")[:m]
    a = _bits(seed, n + m - 1)
    x = _bits(raw, n)
    assert np.array_equal(_karatsuba_hash(a, x, n, m, L, 8), want)
    assert not np.array_equal(_karatsuba_hash(a, x, n, m, L, 8, b_shift=+1), want)
